// Measurement of the plain path's ceiling: the issue rate of the 32 x 32 -> 64-bit
// multiply-add (mad.wide.u32 / IMAD.WIDE.U32) that every modular MAC of the
// s-blocked product costs (Section 5's multiplication phase, one field
// multiply-add per product; here one instruction with lazy 64-bit sums).
//
// Every thread keeps 16 independent 64-bit sums and adds 16 products per
// iteration, as the product kernel's inner loop does; each block stamps its
// SM's cycle counter (clock64) before and after its loop and records its SM.
// The rate per SM is the products of the blocks that ran on that SM over the
// cycles between its first start and its last end, so the result is in
// products per clock per SM, whatever the clock was.
#include <algorithm>
#include <map>
#include <vector>

#include "common.cuh"

namespace pm {

constexpr int PROBE_SUMS = 16;

struct ProbeRec {
    long long start, end;
    int smid, pad;
};

__global__ void mac_probe_kernel(const uint32_t* __restrict__ seed, int64_t iters, uint64_t* __restrict__ sink,
                                 ProbeRec* __restrict__ rec) {
    uint32_t x[PROBE_SUMS];
    uint64_t acc[PROBE_SUMS];
#pragma unroll
    for (int e = 0; e < PROBE_SUMS; ++e) {
        x[e] = seed[(threadIdx.x + e) & 63];
        acc[e] = 0;
    }
    uint32_t y = seed[64 + (threadIdx.x & 63)];
    __syncthreads();
    long long t0 = 0;
    if (threadIdx.x == 0) t0 = clock64();
    // four iterations per trip of a 32-bit loop, so that the loop's own instructions stay
    // a few per 64 products
    const int trips = (int)(iters >> 2);
    for (int it = 0; it < trips; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int e = 0; e < PROBE_SUMS; ++e) acc[e] = mad_wide(x[e], y, acc[e]);
            y += 0x9e3779b9u;  // new products every iteration (one add per 16 products)
        }
    }
    __syncthreads();
    uint64_t t = 0;
#pragma unroll
    for (int e = 0; e < PROBE_SUMS; ++e) t ^= acc[e];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;  // keeps the sums alive
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        rec[blockIdx.x].start = t0;
        rec[blockIdx.x].end = clock64();
        rec[blockIdx.x].smid = (int)smid;
    }
}

}  // namespace pm

using namespace pm;

extern "C" pm_status polymul_probe_mac_rate(int threads, int blocks_per_sm, int64_t iters, double* macs_per_clk_sm,
                                            void* stream) {
    if (!macs_per_clk_sm || threads < 32 || threads > 1024 || threads % 32 || blocks_per_sm < 1 ||
        blocks_per_sm > 32 || iters < 4 || iters > ((int64_t)1 << 32))
        return PM_ERR_INVALID_ARG;
    if (is_capturing(stream)) return PM_ERR_UNSUPPORTED;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    const int nblk = sms * blocks_per_sm;
    const size_t seed_bytes = 128 * sizeof(uint32_t);
    const size_t sink_bytes = (size_t)nblk * threads * sizeof(uint64_t);
    const size_t rec_bytes = (size_t)nblk * sizeof(ProbeRec);
    void* buf = nullptr;
    if (dev_alloc(&buf, seed_bytes + sink_bytes + rec_bytes) != cudaSuccess) {
        cudaGetLastError();
        return PM_ERR_NOMEM;
    }
    uint32_t h_seed[128];
    for (int i = 0; i < 128; ++i) h_seed[i] = 0x12345u * (uint32_t)(i + 1) + 0x6789u;
    uint32_t* d_seed = reinterpret_cast<uint32_t*>(buf);
    uint64_t* d_sink = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(buf) + seed_bytes);
    ProbeRec* d_rec = reinterpret_cast<ProbeRec*>(reinterpret_cast<char*>(buf) + seed_bytes + sink_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    pm_status rc = PM_OK;
    std::vector<ProbeRec> h_rec((size_t)nblk);
    e = cudaMemcpyAsync(d_seed, h_seed, seed_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        mac_probe_kernel<<<nblk, threads, 0, st>>>(d_seed, iters, d_sink, d_rec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_rec.data(), d_rec, rec_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e);
    cudaFree(buf);
    if (rc != PM_OK) return rc;
    count_launches(1);
    // per SM: products of its blocks over the cycles from its first start to its last end
    // (%smid is a physical index and may exceed the SM count, hence the map)
    struct Span {
        long long lo, hi;
        int cnt;
    };
    std::map<int, Span> per_sm;
    for (const ProbeRec& r : h_rec) {
        auto it = per_sm.find(r.smid);
        if (it == per_sm.end()) {
            per_sm[r.smid] = Span{r.start, r.end, 1};
        } else {
            it->second.lo = std::min(it->second.lo, r.start);
            it->second.hi = std::max(it->second.hi, r.end);
            ++it->second.cnt;
        }
    }
    double sum = 0.0;
    int used = 0;
    for (const auto& kv : per_sm) {
        const Span& sp = kv.second;
        if (sp.hi <= sp.lo) continue;
        sum += (double)sp.cnt * threads * (double)(iters / 4 * 4) * PROBE_SUMS / (double)(sp.hi - sp.lo);
        ++used;
    }
    if (!used) return PM_ERR_INTERNAL;
    *macs_per_clk_sm = sum / used;  // the mean over the SMs that ran blocks
    return PM_OK;
}

extern "C" pm_status polymul_probe_mma(int kind, int64_t iters, double* flops_per_clk_sm, int* exact, void* stream) {
    if (!flops_per_clk_sm || !exact || (kind != PM_MMA_BF16 && kind != PM_MMA_E4M3) || iters < 1 ||
        iters > (1 << 20))
        return PM_ERR_INVALID_ARG;
    if (is_capturing(stream)) return PM_ERR_UNSUPPORTED;
    pm_status rc = PM_OK;
    DeviceWorkspace* ws = workspace(stream, &rc);
    if (!ws) return rc;
    return launch_mma_probe(kind, iters, flops_per_clk_sm, exact, (cudaStream_t)stream, ws);
}
