// The s-blocked plain product (Section 5, Algorithms 5-7) on GB300 CUDA cores.
//
// Paper -> this file
//   Algorithm 6 (MulKer): a thread-block copies s coefficients of b and a
//   window of a to local memory and each thread forms s results, each a
//   length-s dot product, written to the auxiliary array M.
//   Algorithm 7 (AddKer): log2(m/s)+1 kernel launches add the rows of M
//   pairwise into f.
// Here one kernel does both phases.  Lane l of a warp owns the s consecutive
// outputs d0 + s*l + e (e < s) of a tile of 32*s outputs.  Per sub-step it
// takes KB = min(s, 8) coefficients of b (a broadcast shared-memory read) and
// forms the s x KB block of products a[d-j] b[j] from a register window of
// s+KB-1 coefficients of a that slides by KB per sub-step; the row sums that
// the paper writes to M stay in 64-bit registers (the multiplication phase),
// and the addition phase is the running sum itself plus two reductions: the 8
// warps of a CTA split the b-range of the tile and add their partial sums in
// shared memory, and up to 8 CTAs of a thread-block cluster split it further
// and add through distributed shared memory.  M never reaches global memory.
//
// Staging (the paper's copy to local memory): per chunk of at most
// CHUNK_MAX coefficients of b, the chunk and the a-window it meets
// (32*s + chunk - 1 coefficients, zero outside [0, n)) are copied with
// coalesced loads into shared memory; a is stored with one pad word every
// 32 (s <= 32) or 64 words so that the 32 lanes' window loads, s words
// apart, hit 32 different banks.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace pm {

constexpr int WB = 8;              // warps per CTA, all on one output tile
constexpr int NT = 32 * WB;        // threads per CTA
constexpr int CHUNK_MAX = 2048;    // b coefficients staged per chunk

template <int S>
struct Cfg {
    static constexpr int KB = S < 8 ? S : 8;     // b coefficients per sub-step
    static constexpr int WIN = S + KB - 1;        // a-window registers per lane
    static constexpr int TD = 32 * S;             // outputs per tile
    static constexpr int PADSH = S > 32 ? 6 : 5;  // one pad word per 2^PADSH words
    static constexpr int A_WORDS = TD + CHUNK_MAX - 1 + ((TD + CHUNK_MAX) >> PADSH) + 4;
    static constexpr int PSTRIDE = TD + 32;       // row of the per-warp partial sums
    static constexpr size_t SMEM =
        sizeof(uint32_t) * (size_t)(((A_WORDS + 3) & ~3) + CHUNK_MAX + WB * PSTRIDE + TD);
};

__device__ __forceinline__ int padded(int i, int sh) { return i + (i >> sh); }

struct Smem {
    uint32_t* sA;
    uint32_t* sB;
    uint32_t* part;
    uint32_t* red;
};

template <int S>
__device__ __forceinline__ Smem carve(uint32_t* base) {
    using C = Cfg<S>;
    Smem s;
    s.sA = base;
    s.sB = s.sA + ((C::A_WORDS + 3) & ~3);
    s.part = s.sB + CHUNK_MAX;
    s.red = s.part + WB * C::PSTRIDE;
    return s;
}

// Multiplication phase of one tile: acc[e] = sum over j in [jb0, jb1) of
// a[d - j] * b[j] for d = d0 + S*lane + e, with a taken as zero outside
// [0, n).  Values are congruent mod p and below 2^64 (see ModParams).
template <int S>
__device__ __forceinline__ void tile_accumulate(const uint32_t* __restrict__ a, int n,
                                                const uint32_t* __restrict__ b, int d0, int jb0,
                                                int jb1, const ModParams& mp, const Smem& sm,
                                                uint64_t (&acc)[S]) {
    using C = Cfg<S>;
    constexpr int KB = C::KB;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < S; ++e) acc[e] = 0;
    int fold_ctr = 0;
    for (int jc = jb0; jc < jb1; jc += CHUNK_MAX) {
        const int clen = min(CHUNK_MAX, jb1 - jc);
        const int wlen = (((clen + WB - 1) / WB) + 7) & ~7;  // per warp, multiple of 8
        const int CL = wlen * WB;                             // padded chunk, <= CHUNK_MAX
        __syncthreads();                                      // previous chunk fully consumed
        for (int i = threadIdx.x; i < CL; i += NT) sm.sB[i] = (i < clen) ? __ldg(b + jc + i) : 0u;
        const int abase = d0 - (jc + CL - 1);
        const int alen = C::TD + CL - 1;
        for (int i = threadIdx.x; i < alen; i += NT) {
            const int ai = abase + i;
            sm.sA[padded(i, C::PADSH)] = (ai >= 0 && ai < n) ? __ldg(a + ai) : 0u;
        }
        __syncthreads();

        const int r0 = warp * wlen;
        int base = S * lane + CL - KB - r0;  // sA index of window slot 0 at sub-step r0
        uint32_t w[C::WIN];
#pragma unroll
        for (int t = 0; t < C::WIN; ++t) w[t] = sm.sA[padded(base + t, C::PADSH)];
        for (int q = 0; q < wlen; q += KB) {
            uint32_t bv[KB];
            if constexpr (KB >= 4) {
#pragma unroll
                for (int k4 = 0; k4 < KB; k4 += 4) {
                    const uint4 v = *reinterpret_cast<const uint4*>(sm.sB + r0 + q + k4);
                    bv[k4] = v.x; bv[k4 + 1] = v.y; bv[k4 + 2] = v.z; bv[k4 + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int k = 0; k < KB; ++k) bv[k] = sm.sB[r0 + q + k];
            }
#pragma unroll
            for (int k = 0; k < KB; ++k) {
#pragma unroll
                for (int e = 0; e < S; ++e) acc[e] = mad_wide(w[e - k + KB - 1], bv[k], acc[e]);
            }
            if (++fold_ctr == mp.fold_every) {
                fold_ctr = 0;
#pragma unroll
                for (int e = 0; e < S; ++e) acc[e] = fold2(acc[e], mp.c32);
            }
            if (q + KB < wlen) {  // slide the window by KB towards lower a indices
#pragma unroll
                for (int t = C::WIN - 1; t >= KB; --t) w[t] = w[t - KB];
                base -= KB;
#pragma unroll
                for (int t = 0; t < KB; ++t) w[t] = sm.sA[padded(base + t, C::PADSH)];
            }
        }
    }
}

// Addition phase inside the CTA: every warp reduces its sums mod p, then the
// 8 partial sums of each output are added.  Leaves red[o] in [0, p).
template <int S>
__device__ __forceinline__ void cta_reduce(uint64_t (&acc)[S], const ModParams& mp,
                                           const Smem& sm) {
    using C = Cfg<S>;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < S; ++e)
        sm.part[warp * C::PSTRIDE + (S + 1) * lane + e] =
            barrett(fold2(acc[e], mp.c32), mp.p, mp.mu);
    __syncthreads();
    for (int o = threadIdx.x; o < C::TD; o += NT) {
        uint64_t s = 0;
#pragma unroll
        for (int w = 0; w < WB; ++w) s += sm.part[w * C::PSTRIDE + o + o / S];
        sm.red[o] = barrett(s, mp.p, mp.mu);
    }
    __syncthreads();
}

// Heavy-first tile order: the middle of the product has the longest sums.
__device__ __forceinline__ int heavy_first(int i, int ntiles) {
    const int mid = (ntiles - 1) / 2;
    const int k = (i + 1) / 2;
    return (i & 1) ? mid + k : mid - k;
}

// One pair; grid = ntiles * cs CTAs in clusters of cs along x.
template <int S>
__global__ void __launch_bounds__(NT) plain_pair_kernel(const uint32_t* __restrict__ a, int n,
                                                        const uint32_t* __restrict__ b, int m,
                                                        uint32_t* __restrict__ c, ModParams mp,
                                                        int ntiles, int cs) {
    using C = Cfg<S>;
    extern __shared__ uint4 smem_raw[];
    const Smem sm = carve<S>(reinterpret_cast<uint32_t*>(smem_raw));
    const int cluster_id = blockIdx.x / cs;
    const int rank = blockIdx.x % cs;
    const int tile = heavy_first(cluster_id, ntiles);
    const int d0 = tile * C::TD;
    const int jlo = max(0, d0 - n + 1);
    const int jhi = min(m, d0 + C::TD);
    const int len = max(0, jhi - jlo);
    const int q = (((len + cs - 1) / cs) + 7) & ~7;
    const int jb0 = min(jhi, jlo + rank * q);
    const int jb1 = min(jhi, jb0 + q);

    uint64_t acc[S];
    tile_accumulate<S>(a, n, b, d0, jb0, jb1, mp, sm, acc);
    cta_reduce<S>(acc, mp, sm);

    const int L = n + m - 1;
    if (cs == 1) {
        for (int o = threadIdx.x; o < C::TD; o += NT)
            if (d0 + o < L) c[d0 + o] = sm.red[o];
        return;
    }
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();  // every CTA's red[] is complete and visible cluster-wide
    const int per = C::TD / cs;
    for (int o = rank * per + threadIdx.x; o < (rank + 1) * per; o += NT) {
        uint64_t s = 0;
        for (int r = 0; r < cs; ++r) s += *cluster.map_shared_rank(sm.red + o, r);
        if (d0 + o < L) c[d0 + o] = barrett(s, mp.p, mp.mu);
    }
    cluster.sync();  // no CTA leaves while another still reads its shared memory
}

// ---------------------------------------------------------------------------
// Batched form: a planner kernel builds a heavy-first work list of
// (pair, output tile) items on the device; a persistent kernel takes items
// through one atomic counter.  Both are stream-ordered, so the pair can be
// captured in a CUDA graph.
// ---------------------------------------------------------------------------
constexpr int PLAN_THREADS = 1024;
constexpr int SORT_MAX = 16384;     // pairs sorted by cost in shared memory

struct BatchWs {
    unsigned int* ctl;   // [0] next item, [1] item count
    int* order;          // pair index of each sorted position
    int64_t* start;      // first item of each sorted position (batch + 1 entries)
};

static size_t batch_ws_bytes(int64_t batch) {
    return 256 + sizeof(int) * (size_t)((batch + 63) & ~63) + sizeof(int64_t) * (size_t)(batch + 1);
}

static BatchWs carve_batch_ws(void* base, int64_t batch) {
    BatchWs w;
    w.ctl = reinterpret_cast<unsigned int*>(base);
    w.order = reinterpret_cast<int*>(reinterpret_cast<char*>(base) + 256);
    w.start = reinterpret_cast<int64_t*>(w.order + ((batch + 63) & ~63));
    return w;
}

__device__ __forceinline__ bool pair_dims(int i, const int64_t* a_off, const int64_t* b_off,
                                          const int64_t* c_off, int64_t max_deg, int64_t* n,
                                          int64_t* m) {
    const int64_t nn = a_off[i + 1] - a_off[i];
    const int64_t mm = b_off[i + 1] - b_off[i];
    const int64_t ll = c_off[i + 1] - c_off[i];
    *n = nn;
    *m = mm;
    return nn >= 1 && mm >= 1 && nn - 1 <= max_deg && mm - 1 <= max_deg && ll == nn + mm - 1 &&
           a_off[i] >= 0 && b_off[i] >= 0 && c_off[i] >= 0;
}

__global__ void __launch_bounds__(PLAN_THREADS) batch_plan_kernel(
    int batch, const int64_t* __restrict__ a_off, const int64_t* __restrict__ b_off,
    const int64_t* __restrict__ c_off, int64_t max_deg, int td, int sort, BatchWs ws,
    int* status) {
    extern __shared__ unsigned long long keys[];
    __shared__ long long s_scan[PLAN_THREADS];
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    int pow2 = 1;
    while (pow2 < batch) pow2 <<= 1;
    // 1. validate, and build sort keys (cost descending, then index ascending)
    for (int i = tid; i < (sort ? pow2 : batch); i += PLAN_THREADS) {
        if (i < batch) {
            int64_t n, m;
            if (!pair_dims(i, a_off, b_off, c_off, max_deg, &n, &m)) s_bad = 1;
            if (sort) {
                unsigned long long cost = (unsigned long long)n * (unsigned long long)m;
                if (cost > 0xFFFFFFFFFFull) cost = 0xFFFFFFFFFFull;
                keys[i] = ((0xFFFFFFFFFFull - cost) << 24) | (unsigned long long)i;
            }
        } else {
            keys[i] = ~0ull;
        }
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            atomicCAS(status, 0, (int)PM_ERR_INVALID_ARG);
            ws.ctl[0] = 0;
            ws.ctl[1] = 0;
        }
        return;
    }
    // 2. bitonic sort of the keys (ascending = heaviest first)
    if (sort) {
        for (int k = 2; k <= pow2; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < pow2; i += PLAN_THREADS) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const unsigned long long x = keys[i], y = keys[ixj];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) { keys[i] = y; keys[ixj] = x; }
                    }
                }
                __syncthreads();
            }
        }
    }
    // 3. exclusive scan of tile counts in sorted order (blocked: each thread a run)
    const int per = (batch + PLAN_THREADS - 1) / PLAN_THREADS;
    const int lo = min(batch, tid * per), hi = min(batch, lo + per);
    long long run = 0;
    for (int k = lo; k < hi; ++k) {
        const int i = sort ? (int)(keys[k] & 0xFFFFFF) : k;
        int64_t n, m;
        pair_dims(i, a_off, b_off, c_off, max_deg, &n, &m);
        run += (n + m - 1 + td - 1) / td;
    }
    s_scan[tid] = run;
    __syncthreads();
    for (int off = 1; off < PLAN_THREADS; off <<= 1) {
        const long long v = tid >= off ? s_scan[tid - off] : 0;
        __syncthreads();
        s_scan[tid] += v;
        __syncthreads();
    }
    long long pos = s_scan[tid] - run;
    for (int k = lo; k < hi; ++k) {
        const int i = sort ? (int)(keys[k] & 0xFFFFFF) : k;
        int64_t n, m;
        pair_dims(i, a_off, b_off, c_off, max_deg, &n, &m);
        ws.order[k] = i;
        ws.start[k] = pos;
        pos += (n + m - 1 + td - 1) / td;
    }
    if (tid == PLAN_THREADS - 1) {
        ws.start[batch] = s_scan[PLAN_THREADS - 1];
        ws.ctl[0] = 0;
        const long long total = s_scan[PLAN_THREADS - 1];
        ws.ctl[1] = total > 0x7FFFFFFF ? 0u : (unsigned int)total;
        if (total > 0x7FFFFFFF) atomicCAS(status, 0, (int)PM_ERR_RANGE);
    }
}

template <int S>
__global__ void __launch_bounds__(NT) plain_batched_kernel(
    int batch, const uint32_t* __restrict__ a_data, const int64_t* __restrict__ a_off,
    const uint32_t* __restrict__ b_data, const int64_t* __restrict__ b_off,
    uint32_t* __restrict__ c_data, const int64_t* __restrict__ c_off, ModParams mp, BatchWs ws) {
    using C = Cfg<S>;
    extern __shared__ uint4 smem_raw[];
    const Smem sm = carve<S>(reinterpret_cast<uint32_t*>(smem_raw));
    __shared__ int s_item;
    const unsigned int total = *(volatile unsigned int*)&ws.ctl[1];
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&ws.ctl[0], 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if ((unsigned int)item >= total) break;
        // sorted position k: the last k with start[k] <= item
        int lo = 0, hi = batch;  // start[lo] <= item < start[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ws.start[mid] <= item) lo = mid; else hi = mid;
        }
        const int pair = ws.order[lo];
        const int tile = (int)(item - ws.start[lo]);
        int n = (int)(a_off[pair + 1] - a_off[pair]);
        int m = (int)(b_off[pair + 1] - b_off[pair]);
        const uint32_t* a = a_data + a_off[pair];
        const uint32_t* b = b_data + b_off[pair];
        if (n < m) {  // the longer operand slides through the window
            const uint32_t* t = a; a = b; b = t;
            const int tn = n; n = m; m = tn;
        }
        const int d0 = tile * C::TD;
        const int jlo = max(0, d0 - n + 1);
        const int jhi = min(m, d0 + C::TD);
        uint64_t acc[S];
        tile_accumulate<S>(a, n, b, d0, jlo, jhi, mp, sm, acc);
        cta_reduce<S>(acc, mp, sm);
        const int L = n + m - 1;
        uint32_t* c = c_data + c_off[pair];
        for (int o = threadIdx.x; o < C::TD; o += NT)
            if (d0 + o < L) c[d0 + o] = sm.red[o];
    }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
template <int S>
static pm_status launch_pair_s(const uint32_t* a, int n, const uint32_t* b, int m, uint32_t* c,
                               uint32_t p, cudaStream_t st, const DeviceWorkspace* ws) {
    using C = Cfg<S>;
    auto kern = plain_pair_kernel<S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e);
    int occ = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e);
    occ = std::max(occ, 1);
    const int L = n + m - 1;
    const int ntiles = (L + C::TD - 1) / C::TD;
    const int want = 2 * ws->num_sms * occ;
    int cs = 1;
    while (cs < 8 && ntiles * cs < want && (std::min(n, m) / (cs * 2)) >= 256) cs *= 2;
    const ModParams mp = host_mod_params(p, C::KB);

    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)(ntiles * cs));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, a, n, b, m, c, mp, ntiles, cs);
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(1);
    return PM_OK;
}

pm_status launch_plain(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* c,
                       uint32_t p, int s, cudaStream_t st, const DeviceWorkspace* ws) {
    if (n < m) {  // the longer operand slides through the window
        std::swap(a, b);
        std::swap(n, m);
    }
    const int ni = (int)n, mi = (int)m;
    switch (s) {
        case 1: return launch_pair_s<1>(a, ni, b, mi, c, p, st, ws);
        case 2: return launch_pair_s<2>(a, ni, b, mi, c, p, st, ws);
        case 4: return launch_pair_s<4>(a, ni, b, mi, c, p, st, ws);
        case 8: return launch_pair_s<8>(a, ni, b, mi, c, p, st, ws);
        case 16: return launch_pair_s<16>(a, ni, b, mi, c, p, st, ws);
        case 32: return launch_pair_s<32>(a, ni, b, mi, c, p, st, ws);
        case 64: return launch_pair_s<64>(a, ni, b, mi, c, p, st, ws);
        default: return PM_ERR_INVALID_ARG;
    }
}

template <int S>
static pm_status launch_batched_s(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                                  const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                                  const int64_t* c_off, uint32_t p, int64_t max_deg,
                                  cudaStream_t st, DeviceWorkspace* ws) {
    using C = Cfg<S>;
    pm_status rc = ensure_buffer(&ws->batch_ws, &ws->batch_ws_bytes, batch_ws_bytes(batch), st);
    if (rc != PM_OK) return rc;
    const BatchWs bw = carve_batch_ws(ws->batch_ws, batch);
    const int sort = batch <= SORT_MAX ? 1 : 0;
    size_t plan_smem = 0;
    if (sort) {
        size_t pow2 = 1;
        while ((int64_t)pow2 < batch) pow2 <<= 1;
        plan_smem = pow2 * sizeof(unsigned long long);
    }
    cudaError_t e = cudaFuncSetAttribute(batch_plan_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<size_t>(plan_smem, 1));
    if (e != cudaSuccess) return cuda_fail(e);
    batch_plan_kernel<<<1, PLAN_THREADS, plan_smem, st>>>((int)batch, a_off, b_off, c_off,
                                                          max_deg, C::TD, sort, bw, ws->status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);

    auto kern = plain_batched_kernel<S>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e);
    int occ = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, C::SMEM);
    if (e != cudaSuccess) return cuda_fail(e);
    occ = std::max(occ, 1);
    const ModParams mp = host_mod_params(p, C::KB);
    kern<<<ws->num_sms * occ, NT, C::SMEM, st>>>((int)batch, a_data, a_off, b_data, b_off, c_data,
                                                 c_off, mp, bw);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(2);
    return PM_OK;
}

pm_status launch_batched_plain(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                               const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                               const int64_t* c_off, uint32_t p, int s, int64_t max_deg,
                               cudaStream_t st, DeviceWorkspace* ws) {
    switch (s) {
#define PM_CASE(SV) \
    case SV:        \
        return launch_batched_s<SV>(batch, a_data, a_off, b_data, b_off, c_data, c_off, p, max_deg, st, ws);
        PM_CASE(1) PM_CASE(2) PM_CASE(4) PM_CASE(8) PM_CASE(16) PM_CASE(32) PM_CASE(64)
#undef PM_CASE
        default: return PM_ERR_INVALID_ARG;
    }
}

}  // namespace pm
