// The batched product from host buffers (polymul_batched_host): the batch is
// cut into chunks of consecutive pairs, and each chunk's words travel to the
// device, are multiplied by polymul_batched and travel back on three streams
// of the library's own, so that the copy of chunk k + 1 to the device, the
// product of chunk k and the copy of chunk k - 1 back to the host overlap.
// Two device slots (inputs, products, offsets) alternate between the chunks;
// events order each slot's reuse after the work that last used it.  The
// offsets of a chunk are copied as they are and rebased on the device (a
// kernel subtracts the chunk's first offset), so the host only reads the
// three offsets that bound each chunk.
//
// The paper has no host-to-device path; this is the end-to-end form of the
// batched product.
#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace pm {

// chunk weights (shares of the batch's multiply-adds): the first chunk's upload and the last
// one's download are the only copies no product hides, so those chunks are the lightest
// (1024 pairs of degree 4095 from pinned buffers, ms: 1:3:3:1 0.633; four equal chunks 0.677;
// eight 0.753; 1:2:2:2:1 0.660)
constexpr int HIO_CHUNKS = 4;
constexpr int HIO_W[HIO_CHUNKS] = {1, 3, 3, 1};

struct HostIoSlot {
    void* buf = nullptr;
    size_t bytes = 0;
};

struct HostIo {
    cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
    cudaEvent_t ev_start = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {};
    HostIoSlot slot[2];
    bool used[2] = {false, false};
};

static std::mutex g_hio_mutex;
static HostIo* g_hio[64] = {};

// off[i] -= base for the chunk's three offset arrays (k + 1 entries each)
__global__ void hio_rebase_kernel(int64_t* __restrict__ off, int64_t k1, int64_t base_a, int64_t base_b,
                                  int64_t base_c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * k1) return;
    off[i] -= i < k1 ? base_a : (i < 2 * k1 ? base_b : base_c);
}

static pm_status hio_state(int dev, HostIo** out) {
    if (g_hio[dev]) {
        *out = g_hio[dev];
        return PM_OK;
    }
    HostIo* h = new HostIo();
    cudaError_t e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&h->ev_in[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_comp[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out[b], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e);  // (the handles created so far are kept by the process)
    g_hio[dev] = h;
    *out = h;
    return PM_OK;
}

void release_host_io() {
    std::lock_guard<std::mutex> lock(g_hio_mutex);
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < 64; ++d) {
        HostIo* h = g_hio[d];
        if (!h) continue;
        cudaSetDevice(d);
        cudaStreamSynchronize(h->s_in);
        cudaStreamSynchronize(h->s_comp);
        cudaStreamSynchronize(h->s_out);
        for (int b = 0; b < 2; ++b) {
            if (h->slot[b].buf) cudaFree(h->slot[b].buf);
            cudaEventDestroy(h->ev_in[b]);
            cudaEventDestroy(h->ev_comp[b]);
            cudaEventDestroy(h->ev_out[b]);
        }
        cudaEventDestroy(h->ev_start);
        cudaStreamDestroy(h->s_in);
        cudaStreamDestroy(h->s_comp);
        cudaStreamDestroy(h->s_out);
        delete h;
        g_hio[d] = nullptr;
    }
    cudaSetDevice(cur);
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace pm

using namespace pm;

extern "C" pm_status polymul_batched_host(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                                          const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                                          const int64_t* c_off, uint32_t p, int mode, int s, int64_t max_deg,
                                          void* stream) {
    if (batch < 0 || batch > (int64_t)(1 << 24)) return PM_ERR_INVALID_ARG;
    if (batch == 0) return PM_OK;
    if (!a_data || !a_off || !b_data || !b_off || !c_data || !c_off) return PM_ERR_INVALID_ARG;
    if (max_deg < 0 || max_deg > PM_MAX_DEG) return PM_ERR_INVALID_ARG;
    if (p < 2 || p >= PM_MAX_P) return PM_ERR_RANGE;
    if (mode != PM_AUTO && mode != PM_PLAIN && mode != PM_TENSOR) return PM_ERR_INVALID_ARG;
    if (mode == PM_TENSOR && !(p < (1u << 29) && max_deg <= PM_TENSOR_MAX_DEG)) return PM_ERR_UNSUPPORTED;
    // the host offsets bound the words each chunk copies: check them here (the device planners
    // check every pair again)
    for (int64_t i = 0; i < batch; ++i) {
        const int64_t n = a_off[i + 1] - a_off[i], m = b_off[i + 1] - b_off[i];
        if (a_off[i] < 0 || b_off[i] < 0 || c_off[i] < 0 || n < 1 || m < 1 || n - 1 > max_deg ||
            m - 1 > max_deg || c_off[i + 1] - c_off[i] != n + m - 1)
            return PM_ERR_INVALID_ARG;
    }
    // the products must not land on the inputs (later chunks still read them)
    auto apart = [](const void* x, size_t xb, const void* y, size_t yb) {
        const char *cx = static_cast<const char*>(x), *cy = static_cast<const char*>(y);
        return cx + xb <= cy || cy + yb <= cx;
    };
    const size_t cb = 4 * (size_t)c_off[batch];
    if (!apart(c_data, cb, a_data, 4 * (size_t)a_off[batch]) || !apart(c_data, cb, b_data, 4 * (size_t)b_off[batch]))
        return PM_ERR_INVALID_ARG;
    if (is_capturing(stream)) return PM_ERR_UNSUPPORTED;
    pm_status rc = PM_OK;
    DeviceWorkspace* ws = workspace(stream, &rc);
    if (!ws) return rc;
    std::lock_guard<std::mutex> lock(g_hio_mutex);
    HostIo* h = nullptr;
    if ((rc = hio_state(ws->device, &h)) != PM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    // chunk bounds: shares of the batch's multiply-adds in the proportions HIO_W (equal shares when
    // the batch has fewer pairs than chunks)
    const int nch = (int)std::min<int64_t>(HIO_CHUNKS, batch);
    std::vector<double> frac(nch + 1, 0.0);
    {
        double wsum = 0.0;
        for (int k = 0; k < nch; ++k) wsum += nch == HIO_CHUNKS ? HIO_W[k] : 1.0;
        for (int k = 0; k < nch; ++k) frac[k + 1] = frac[k] + (nch == HIO_CHUNKS ? HIO_W[k] : 1.0) / wsum;
    }
    std::vector<int64_t> cut(nch + 1, batch);
    {
        double tot = 0.0;
        for (int64_t i = 0; i < batch; ++i) tot += (double)(a_off[i + 1] - a_off[i]) * (double)(b_off[i + 1] - b_off[i]);
        double run = 0.0;
        int k = 1;
        cut[0] = 0;
        for (int64_t i = 0; i < batch && k < nch; ++i) {
            run += (double)(a_off[i + 1] - a_off[i]) * (double)(b_off[i + 1] - b_off[i]);
            if (run >= tot * frac[k] && i + 1 < batch) cut[k++] = i + 1;
        }
        for (; k < nch; ++k) cut[k] = std::max(cut[k - 1], std::min<int64_t>(batch, cut[k - 1] + 1));
        cut[nch] = batch;
    }
    // a slot holds one chunk in regions of fixed place for the call (sized for the largest chunk):
    // a words | b words | c words | 3 (k + 1) offsets.  The copies of a chunk's inputs then never
    // touch the products region that the copy of the slot's previous chunk back to the host reads.
    size_t max_a = 0, max_b = 0, max_c = 0, max_k = 0;
    for (int k = 0; k < nch; ++k) {
        const int64_t p0 = cut[k], p1 = cut[k + 1];
        max_a = std::max(max_a, (size_t)(a_off[p1] - a_off[p0]));
        max_b = std::max(max_b, (size_t)(b_off[p1] - b_off[p0]));
        max_c = std::max(max_c, (size_t)(c_off[p1] - c_off[p0]));
        max_k = std::max(max_k, (size_t)(p1 - p0 + 1));
    }
    const size_t off_b = align256(4 * max_a), off_c = off_b + align256(4 * max_b);
    const size_t off_o = off_c + align256(4 * max_c);
    const size_t need = off_o + 3 * 8 * max_k;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2; ++b) {
        if (h->slot[b].bytes >= need) continue;
        // a slot grows only after the work that used it is done
        if (h->used[b]) {
            e = cudaStreamSynchronize(h->s_in);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->s_comp);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->s_out);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        if (h->slot[b].buf) cudaFree(h->slot[b].buf);
        h->slot[b].buf = nullptr;
        h->slot[b].bytes = 0;
        size_t want = 1 << 20;
        while (want < need) want *= 2;
        if (dev_alloc(&h->slot[b].buf, want) != cudaSuccess) {
            cudaGetLastError();
            return PM_ERR_NOMEM;
        }
        h->slot[b].bytes = want;
        h->used[b] = false;
    }
    // the copies to the device start after the work queued before the call on `stream`
    e = cudaEventRecord(h->ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_in, h->ev_start, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int k = 0; k < nch; ++k) {
        const int b = k & 1;
        const int64_t p0 = cut[k], p1 = cut[k + 1], kp = p1 - p0;
        const size_t na = (size_t)(a_off[p1] - a_off[p0]), nb = (size_t)(b_off[p1] - b_off[p0]);
        const size_t nc = (size_t)(c_off[p1] - c_off[p0]);
        char* base = static_cast<char*>(h->slot[b].buf);
        uint32_t* da = reinterpret_cast<uint32_t*>(base);
        uint32_t* db = reinterpret_cast<uint32_t*>(base + off_b);
        uint32_t* dc = reinterpret_cast<uint32_t*>(base + off_c);
        int64_t* doff = reinterpret_cast<int64_t*>(base + off_o);
        // inputs: after the slot's previous product (which read them) is done, and after the copy
        // of its products back to the host (a call's layout differs from the previous call's)
        if (h->used[b]) e = cudaStreamWaitEvent(h->s_in, h->ev_comp[b], 0);
        if (e == cudaSuccess && h->used[b] && k < 2) e = cudaStreamWaitEvent(h->s_in, h->ev_out[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(da, a_data + a_off[p0], 4 * na, cudaMemcpyHostToDevice, h->s_in);
        if (e == cudaSuccess) e = cudaMemcpyAsync(db, b_data + b_off[p0], 4 * nb, cudaMemcpyHostToDevice, h->s_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(doff, a_off + p0, 8 * (kp + 1), cudaMemcpyHostToDevice, h->s_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(doff + (kp + 1), b_off + p0, 8 * (kp + 1), cudaMemcpyHostToDevice, h->s_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(doff + 2 * (kp + 1), c_off + p0, 8 * (kp + 1), cudaMemcpyHostToDevice, h->s_in);
        if (e == cudaSuccess) {
            const int64_t words = 3 * (kp + 1);
            hio_rebase_kernel<<<(unsigned)((words + 255) / 256), 256, 0, h->s_in>>>(doff, kp + 1, a_off[p0],
                                                                                 b_off[p0], c_off[p0]);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[b], h->s_in);
        // product: after the inputs, and after the slot's previous products went back to the host
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_comp, h->ev_in[b], 0);
        if (e == cudaSuccess && h->used[b]) e = cudaStreamWaitEvent(h->s_comp, h->ev_out[b], 0);
        if (e != cudaSuccess) return cuda_fail(e);
        count_launches(1);
        rc = polymul_batched(kp, da, doff, db, doff + (kp + 1), dc, doff + 2 * (kp + 1), p, mode, s, max_deg,
                             (void*)h->s_comp);
        if (rc != PM_OK) return rc;
        e = cudaEventRecord(h->ev_comp[b], h->s_comp);
        // products back to the host
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->ev_comp[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c_data + c_off[p0], dc, 4 * nc, cudaMemcpyDeviceToHost, h->s_out);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[b], h->s_out);
        if (e != cudaSuccess) return cuda_fail(e);
        h->used[b] = true;
    }
    // `stream` goes on once every product is back on the host
    e = cudaStreamWaitEvent(st, h->ev_out[(nch - 1) & 1], 0);
    if (e != cudaSuccess) return cuda_fail(e);
    return PM_OK;
}
