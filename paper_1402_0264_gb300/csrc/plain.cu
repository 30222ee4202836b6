// The s-blocked plain product (Section 5, Algorithms 5-7) on GB300 CUDA cores.
//
// Paper -> this file
//   Algorithm 6 (MulKer): a thread-block copies s coefficients of b and a
//   window of a to local memory; each thread forms s results, each a
//   length-s dot product, and writes them to the auxiliary array M.
//   Algorithm 7 (AddKer): log2(m/s)+1 launches add the rows of M pairwise.
// Here both phases run in one persistent kernel and M never reaches global
// memory.  Lane l of a warp owns the s consecutive outputs d0 + s*l + e
// (e < s) of a tile of 32*s outputs.  Per sub-step it takes KB = min(s, 8)
// coefficients of b (one broadcast shared-memory read) and forms the s x KB
// block of products a[d-j] b[j] from a register window of s+KB-1 coefficients
// of a, kept as a ring of KB-word groups that slides by one group per
// sub-step (so no register moves).  Row sums stay in 64-bit registers: that is
// the multiplication phase with the first levels of the addition phase fused
// into it.  The 8 warps of a CTA split the b-range of a tile and add their
// partial sums in shared memory.
//
// Work distribution.  The paper's kernels are grids of independent blocks;
// with one CTA per output tile the largest tiles finish last and the SMs idle
// (a tail of about one tile).  Instead every tile t of every pair is cut into
// len(t) "positions", one per coefficient of b that meets the tile (len(t) =
// min(m, (t+1)T) - max(0, tT - n + 1) for T = 32 s outputs per tile, with a
// the longer operand), and the G positions of the whole job are split into P
// equal contiguous ranges, one per persistent CTA.  A tile covered by one CTA
// is written directly; a tile cut by CTA boundaries gets one partial sum per
// CTA in a scratch slot, and the CTA that arrives last at the tile's counter
// adds them and writes the output (the counter is reset by that CTA, so the
// scratch is clean for the next call).  No CTA ever waits for another.
//
// Staging (the paper's copy to local memory): per chunk of at most
// CHUNK_MAX coefficients of b, the chunk and the a-window it meets
// (32*s + chunk - 1 coefficients, zero outside [0, n)) are copied with
// coalesced loads into shared memory.  The a-window is stored in 16-byte
// chunks with one pad chunk after every 8, so that the 32 lanes' 128-bit
// window loads (s words apart) fall in distinct banks for s = 4..32.
#include <algorithm>

#include "common.cuh"

namespace pm {

#ifndef PM_WB
#define PM_WB 8
#endif
constexpr int WB = PM_WB;        // warps per CTA, all on one output tile
constexpr int NT = 32 * WB;      // threads per CTA
constexpr int CHUNK_MAX = 2048;  // b coefficients staged per chunk (two chunks in flight)
constexpr int FRONT = 8;         // a-window words before index 0 (read by the last prefetch)
constexpr int FIRST_CHUNK = 512; // a CTA's very first chunk: short, so that its products start early

// Build-time tuning knobs (defaults chosen by measurement on GB300).
#ifndef PM_MINB
#define PM_MINB 0                // __launch_bounds__ minimum blocks per SM (0: none)
#endif
#if PM_MINB > 0
#define PM_BOUNDS(W) __launch_bounds__(32 * (W), PM_MINB)
#else
#define PM_BOUNDS(W) __launch_bounds__(32 * (W))
#endif

// W = warps per CTA (the paper's l = 32 W threads per block); WB by default,
// 4 and 16 for the block-size study (polymul_plain_ell).
template <int S, int W = WB>
struct Cfg {
    static constexpr int KB = S < 8 ? S : 8;                   // b coefficients per sub-step
    static constexpr int NGW = (S + KB - 1 + KB - 1) / KB;     // window groups of KB words
    static constexpr int R = NGW + 1;                          // ring slots (one prefetched)
    static constexpr int TD = 32 * S;                          // outputs per tile
    static constexpr int A_LOGICAL = FRONT + TD + CHUNK_MAX + 8;
    static constexpr int A_CHUNKS = (A_LOGICAL + 3) / 4;
    static constexpr int A_WORDS = 4 * (A_CHUNKS + A_CHUNKS / 8 + 2);
    static constexpr int PSTRIDE = TD + 32;                    // row of per-warp partial sums
    static constexpr int BUF_WORDS = A_WORDS + CHUNK_MAX;       // one staging buffer
    static constexpr size_t SMEM = 4 * (size_t)(2 * BUF_WORDS + W * PSTRIDE + TD);
};

// word offset of logical a-window word i (16-byte chunks, a pad chunk every 8)
__device__ __forceinline__ int a_phys(int i) { return 4 * ((i >> 2) + (i >> 5)) + (i & 3); }

struct Smem {
    uint32_t* buf;   // two staging buffers: a-window (A_WORDS) then b-chunk (CHUNK_MAX)
    uint32_t* part;
    uint32_t* red;
};

template <int S, int W = WB>
__device__ __forceinline__ Smem carve(uint32_t* base) {
    using C = Cfg<S, W>;
    Smem s;
    s.buf = base;
    s.part = s.buf + 2 * C::BUF_WORDS;
    s.red = s.part + W * C::PSTRIDE;
    return s;
}

// 4-byte asynchronous global->shared copy; with valid == false it writes a zero
// and reads nothing (src-size 0), src is then only a placeholder address.
__device__ __forceinline__ void cp_async4(uint32_t* dst, const uint32_t* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Chunk `ci` of the b-range [jb0, jb1), whose chunk 0 holds f coefficients
// and the others CHUNK_MAX: start, length and padded length CL (a multiple of
// KB).  Warp w takes sub-steps [first, first + count) of the CL / KB
// sub-steps, the counts differing by at most one.
struct ChunkDims {
    int jc, clen, CL;
};
template <int KB, int CH = CHUNK_MAX>
__device__ __forceinline__ ChunkDims chunk_dims(int jb0, int jb1, int ci, int f) {
    ChunkDims c;
    c.jc = jb0 + (ci == 0 ? 0 : f + (ci - 1) * CH);
    c.clen = min(ci == 0 ? f : CH, jb1 - c.jc);
    c.CL = (c.clen + KB - 1) / KB * KB;
    return c;
}

// Issues the copies of one chunk: b[jc .. jc+clen) (zeros up to CL) and the
// a-window a[d0-(jc+CL-1) .. d0+TD-jc) (zeros outside [0, n)), by threads
// tid, tid + nthr, ... of the group that stages (AW = a-window words).
template <int S, int AW, int CH = CHUNK_MAX>
__device__ __forceinline__ void stage_chunk(const uint32_t* __restrict__ a, int n,
                                            const uint32_t* __restrict__ b, int m, int d0,
                                            const ChunkDims& ch, uint32_t* buf, int tid, int nthr) {
    using C = Cfg<S>;
    uint32_t* sA = buf;
    uint32_t* sB = buf + AW;
    for (int i = tid; i < ch.CL; i += nthr) {
        const bool v = i < ch.clen;
        if (PM_CHK(i < CH && (!v || (ch.jc + i >= 0 && ch.jc + i < m))))
            cp_async4(sB + i, b + (v ? ch.jc + i : 0), v);
    }
    const int abase = d0 - (ch.jc + ch.CL - 1);
    const int alen = C::TD + ch.CL - 1;
    for (int i = tid; i < alen; i += nthr) {
        const int ai = abase + i;
        const bool v = ai >= 0 && ai < n;
        if (PM_CHK(a_phys(FRONT + i) < AW)) cp_async4(sA + a_phys(FRONT + i), a + (v ? ai : 0), v);
    }
    cp_async_commit();
}

// One group of KB consecutive a-window words starting at window index `base`.
template <int S>
__device__ __forceinline__ void load_group(const uint32_t* sA, int base, uint32_t (&g)[Cfg<S>::KB]) {
    constexpr int KB = Cfg<S>::KB;
    const int li = FRONT + base;
    if constexpr (KB >= 4) {  // li is a multiple of 4 here
#pragma unroll
        for (int h = 0; h < KB / 4; ++h) {
            const int j = (li >> 2) + h;
            const uint4 v = *reinterpret_cast<const uint4*>(sA + 4 * (j + (j >> 3)));
            g[4 * h] = v.x; g[4 * h + 1] = v.y; g[4 * h + 2] = v.z; g[4 * h + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int t = 0; t < KB; ++t) g[t] = sA[a_phys(li + t)];
    }
}

// Multiplication phase of one staged chunk (CL coefficients of b and the
// a-window they meet): acc[e] += sum over the chunk of a[d - j] b[j] for
// d = d0 + S*lane + e, over the share of warp `warp` of the nw warps that
// split the chunk.  Values stay congruent mod p and below 2^64 (see
// ModParams); fold_ctr counts sub-steps since the last fold.
template <int S, int AW = Cfg<S>::A_WORDS, int CH = CHUNK_MAX>
__device__ __forceinline__ void compute_chunk(const uint32_t* sA, const uint32_t* sB, int CL,
                                              const ModParams& mp, uint64_t (&acc)[S], int& fold_ctr,
                                              int warp, int nw) {
    using C = Cfg<S>;
    constexpr int KB = C::KB, NGW = C::NGW, R = C::R;
    const int lane = threadIdx.x & 31;
    const int tot = CL / KB, qw = tot / nw, rw = tot % nw;
    const int nsub = qw + (warp < rw ? 1 : 0);
    const int r0 = KB * (warp * qw + min(warp, rw));
    int base = S * lane + CL - KB - r0;  // window index of group 0 at the current sub-step
    // the window words this thread reads run from base - nsub KB (the last prefetch) to
    // base + NGW KB - 1, the b words from r0 to r0 + nsub KB - 1
    if (!PM_CHK(FRONT + base - nsub * KB >= 0 && a_phys(FRONT + base + NGW * KB - 1) < AW &&
                r0 + nsub * KB <= CH))
        return;
    uint32_t ring[R][KB];
#pragma unroll
    for (int g = 0; g < NGW; ++g) load_group<S>(sA, base + g * KB, ring[(R - g) % R]);
    const uint32_t* bp = sB + r0;
    // sub-step at ring position u (a constant once the loops below are unrolled,
    // so the ring stays in fixed registers)
    auto substep = [&](int u) {
        load_group<S>(sA, base - KB, ring[(u + 1) % R]);  // group 0 of the next sub-step
        uint32_t bv[KB];
        if constexpr (KB >= 4) {
#pragma unroll
            for (int k4 = 0; k4 < KB; k4 += 4) {
                const uint4 v = *reinterpret_cast<const uint4*>(bp + k4);
                bv[k4] = v.x; bv[k4 + 1] = v.y; bv[k4 + 2] = v.z; bv[k4 + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < KB; ++k) bv[k] = bp[k];
        }
#pragma unroll
        for (int k = 0; k < KB; ++k) {
#pragma unroll
            for (int e = 0; e < S; ++e) {
                const int t = e - k + KB - 1;  // window word of a[d - j]
                acc[e] = mad_wide(ring[(u - t / KB + R) % R][t % KB], bv[k], acc[e]);
            }
        }
        base -= KB;
        bp += KB;
    };
    auto fold_all = [&]() {
        fold_ctr = 0;
        if (mp.fold_twice) {
#pragma unroll
            for (int e = 0; e < S; ++e) acc[e] = fold2(acc[e], mp.c32);
        } else {
#pragma unroll
            for (int e = 0; e < S; ++e) acc[e] = fold_once(acc[e], mp.c32);
        }
    };
    int q0 = 0;
    if (mp.fold_every >= R) {
        // whole blocks of R sub-steps, with no test inside: the fold falls due
        // at most once per block and is done before the block if needed
        for (; q0 + R <= nsub; q0 += R) {
            if (fold_ctr + R > mp.fold_every) fold_all();
#pragma unroll
            for (int u = 0; u < R; ++u) substep(u);
            fold_ctr += R;
        }
    }
    // the last nsub mod R sub-steps (all of them when folds are due more often);
    // at most fold_every sub-steps ever separate two folds
    for (; q0 < nsub; q0 += R) {
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (q0 + u < nsub) {
                if (fold_ctr >= mp.fold_every) fold_all();
                substep(u);
                ++fold_ctr;
            }
        }
    }
}

// Addition phase inside the CTA: every warp reduces its sums mod p, then the
// 8 partial sums of each output are added.  Leaves red[o] in [0, p).
template <int S, int W = WB>
__device__ __forceinline__ void cta_reduce(uint64_t (&acc)[S], const ModParams& mp,
                                           const Smem& sm) {
    using C = Cfg<S, W>;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < S; ++e)
        sm.part[warp * C::PSTRIDE + (S + 1) * lane + e] = barrett(fold2(acc[e], mp.c32), mp.p, mp.mu);
    __syncthreads();
    for (int o = threadIdx.x; o < C::TD; o += 32 * W) {
        uint64_t s = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) s += sm.part[w * C::PSTRIDE + o + o / S];
        sm.red[o] = barrett(s, mp.p, mp.mu);
    }
    __syncthreads();
}

// ---- positions: len(t) and its prefix sum in closed form (n >= m >= 1) ----
__host__ __device__ __forceinline__ int64_t ntiles_of(int64_t n, int64_t m, int64_t td) {
    return (n + m - 1 + td - 1) / td;
}

__host__ __device__ __forceinline__ int64_t tile_jlo(int64_t n, int64_t td, int64_t t) {
    const int64_t x = t * td - (n - 1);
    return x > 0 ? x : 0;
}

// sum_{t<T} len(t), len(t) = min(m, (t+1) td) - max(0, t td - (n-1))
__host__ __device__ __forceinline__ int64_t cum_len(int64_t n, int64_t m, int64_t td, int64_t T) {
    int64_t u0 = m / td;
    if (u0 > T) u0 = T;
    const int64_t s1 = td * (u0 * (u0 + 1) / 2) + m * (T - u0);
    const int64_t t1 = (n - 1) / td + 1;
    int64_t s2 = 0;
    if (T > t1) {
        const int64_t cnt = T - t1;
        s2 = td * ((t1 + T - 1) * cnt / 2) - (n - 1) * cnt;
    }
    return s1 - s2;
}

constexpr int64_t MIN_POSITIONS = 64;  // smallest share of a CTA (positions of TD MACs each)
constexpr int64_t COUNTER_REGION_DEV = 32768;  // tile counters at the start of the scratch (COUNTER_REGION)

// Scratch of one launch: 2 partial-sum slots of TD words per CTA and one
// counter per CTA (zero between calls).
struct SkScratch {
    uint32_t* slots;
    unsigned int* counters;
};

// Partition of G positions into P ranges: the first r = G mod P ranges hold
// q + 1 = floor(G / P) + 1 positions, the others q (q >= 1 since P <= G).
struct Split {
    int64_t q, r;
    __device__ __forceinline__ int64_t start(int64_t k) const { return k * q + (k < r ? k : r); }
    // the range holding position x
    __device__ __forceinline__ int64_t owner(int64_t x) const {
        const int64_t big = r * (q + 1);
        return x < big ? x / (q + 1) : r + (x - big) / q;
    }
};

// One segment of a CTA's range: the part [x, x_end) of tile t of one pair.
struct Seg {
    const uint32_t* a;
    const uint32_t* b;
    uint32_t* c;
    int n, m;              // n >= m (the longer operand slides through the window)
    int d0;                // first output of the tile
    int jb0, jb1;          // coefficients of b of this segment
    int f;                 // coefficients in chunk 0
    int nchunks;
    int64_t x, x_end, s_tile, e_tile;  // positions
};

// Walks a CTA's segments in order: pi = current pair, t = tile of the last
// segment in it (-1: not known, search).
template <int S, bool BATCH, int CH = CHUNK_MAX>
__device__ __forceinline__ Seg make_seg(int64_t x, int64_t x1, int& pi, int64_t& t,
                                        const uint32_t* __restrict__ a_data, const int64_t* __restrict__ a_off,
                                        const uint32_t* __restrict__ b_data, const int64_t* __restrict__ b_off,
                                        uint32_t* __restrict__ c_data, const int64_t* __restrict__ c_off,
                                        int n1, int m1, const int64_t* __restrict__ prefix) {
    using C = Cfg<S>;
    Seg sg;
    int64_t pbase = 0;
    if constexpr (BATCH) {
        while (prefix[pi + 1] <= x) { ++pi; t = -1; }
        pbase = prefix[pi];
        sg.a = a_data + a_off[pi];
        sg.b = b_data + b_off[pi];
        sg.c = c_data + c_off[pi];
        sg.n = (int)(a_off[pi + 1] - a_off[pi]);
        sg.m = (int)(b_off[pi + 1] - b_off[pi]);
    } else {
        sg.a = a_data; sg.b = b_data; sg.c = c_data; sg.n = n1; sg.m = m1;
    }
    if (sg.n < sg.m) {
        const uint32_t* tp = sg.a; sg.a = sg.b; sg.b = tp;
        const int tn = sg.n; sg.n = sg.m; sg.m = tn;
    }
    const int64_t nt = ntiles_of(sg.n, sg.m, C::TD);
    if (t >= 0) {
        ++t;  // the previous segment ended with its tile: x starts the next one
    } else {
        const int64_t y = x - pbase;
        int64_t tlo = 0, thi = nt;
        while (thi - tlo > 1) {
            const int64_t mid = (tlo + thi) >> 1;
            if (cum_len(sg.n, sg.m, C::TD, mid) <= y) tlo = mid; else thi = mid;
        }
        t = tlo;
    }
    sg.s_tile = pbase + cum_len(sg.n, sg.m, C::TD, t);
    sg.e_tile = pbase + cum_len(sg.n, sg.m, C::TD, t + 1);
    sg.x = x;
    sg.x_end = x1 < sg.e_tile ? x1 : sg.e_tile;
    const int64_t jlo = tile_jlo(sg.n, C::TD, t);
    sg.d0 = (int)(t * C::TD);
    sg.jb0 = (int)(jlo + (x - sg.s_tile));
    sg.jb1 = (int)(jlo + (sg.x_end - sg.s_tile));
    sg.f = CH;
    sg.nchunks = (sg.jb1 - sg.jb0 + CH - 1) / CH;
    if (t + 1 == nt) t = -1;  // the pair ends with this tile
    return sg;
}

// Addition phase of a finished segment: the CTA's sums, then either the
// tile's outputs (the CTA owns the whole tile) or a partial-sum slot; the CTA
// that brings the tile's counter to its last value adds the slots and writes.
template <int S, int W = WB>
__device__ __forceinline__ void finish_segment(const Seg& sg, uint64_t (&acc)[S], const ModParams& mp,
                                               const Smem& sm, const Split& sp, int64_t k, int64_t x0,
                                               SkScratch sk, int* s_last) {
    using C = Cfg<S, W>;
    constexpr int NTW = 32 * W;
    cta_reduce<S, W>(acc, mp, sm);
    const int L = sg.n + sg.m - 1;
    if (sg.x == sg.s_tile && sg.x_end == sg.e_tile) {
        for (int o = threadIdx.x; o < C::TD; o += NTW)
            if (sg.d0 + o < L) sg.c[sg.d0 + o] = sm.red[o];
        return;
    }
    const int64_t k1 = sp.owner(sg.s_tile), k2 = sp.owner(sg.e_tile - 1);
    const int64_t slot = 2 * k + (sg.x == x0 ? 0 : 1);
    // (the scratch holds 2 slots per launched CTA and COUNTER_REGION counters)
    if (!PM_CHK(slot < 2 * (int64_t)gridDim.x && k1 >= 0 && k2 < (int64_t)gridDim.x && k1 < COUNTER_REGION_DEV))
        return;
    uint32_t* mine = sk.slots + slot * C::TD;
    for (int o = threadIdx.x; o < C::TD; o += NTW) mine[o] = sm.red[o];
    __syncthreads();
    if (threadIdx.x == 0) {
        // the barrier orders every thread's slot writes before this fence, and a
        // fence orders what its thread has observed: the slot is visible before
        // the count is
        __threadfence();
        const unsigned int seen = atomicAdd(&sk.counters[k1], 1u);
        const int last = seen == (unsigned int)(k2 - k1) ? 1 : 0;
        if (last) __threadfence();  // and the other contributors' slots before the reads below
        *s_last = last;
    }
    __syncthreads();
    if (*s_last) {  // every other contributor has written its slot
        const int64_t first_slot = 2 * k1 + (sp.start(k1) == sg.s_tile ? 0 : 1);
        for (int o = threadIdx.x; o < C::TD; o += NTW) {
            // four independent sums keep several L2 reads in flight
            uint64_t s0 = __ldcg(sk.slots + first_slot * C::TD + o), s1 = 0, s2 = 0, s3 = 0;
            int64_t kk = k1 + 1;
            for (; kk + 3 <= k2; kk += 4) {
                s0 += __ldcg(sk.slots + 2 * kk * C::TD + o);
                s1 += __ldcg(sk.slots + 2 * (kk + 1) * C::TD + o);
                s2 += __ldcg(sk.slots + 2 * (kk + 2) * C::TD + o);
                s3 += __ldcg(sk.slots + 2 * (kk + 3) * C::TD + o);
            }
            for (; kk <= k2; ++kk) s0 += __ldcg(sk.slots + 2 * kk * C::TD + o);
            if (sg.d0 + o < L) sg.c[sg.d0 + o] = barrett(s0 + s1 + s2 + s3, mp.p, mp.mu);
        }
        if (threadIdx.x == 0) sk.counters[k1] = 0;
    }
    __syncthreads();  // s_last is read before the next segment may set it
}

// Persistent Stream-K kernel.  BATCH = false: one pair (a, n1, b, m1, c).
// BATCH = true: pair i from the CSR arrays; prefix[i] = positions before pair i.
// The CTA's chunks form one stream across its segments: the next chunk (of
// this segment or the next) is copied in while the current one is used.
template <int S, bool BATCH, int W = WB>
__global__ void PM_BOUNDS(W) plain_sk_kernel(
    const uint32_t* __restrict__ a_data, const int64_t* __restrict__ a_off,
    const uint32_t* __restrict__ b_data, const int64_t* __restrict__ b_off,
    uint32_t* __restrict__ c_data, const int64_t* __restrict__ c_off, int n1, int m1,
    const int64_t* __restrict__ prefix, int batch, ModParams mp, SkScratch sk) {
    using C = Cfg<S, W>;
    constexpr int NTW = 32 * W;
    constexpr int KB = C::KB;
    extern __shared__ uint4 smem_raw[];
    __shared__ int s_last;
    const Smem sm = carve<S, W>(reinterpret_cast<uint32_t*>(smem_raw));
    int64_t G;
    if constexpr (BATCH) {
        G = prefix[batch];
    } else {
        const int64_t nn = n1 >= m1 ? n1 : m1, mm = n1 >= m1 ? m1 : n1;
        G = cum_len(nn, mm, C::TD, ntiles_of(nn, mm, C::TD));
    }
    // CTAs that would get fewer than MIN_POSITIONS positions stay idle
    const int64_t pmax = G / MIN_POSITIONS > 1 ? G / MIN_POSITIONS : 1;
    const int64_t P = pmax < (int64_t)gridDim.x ? pmax : (int64_t)gridDim.x;
    const int64_t k = blockIdx.x;
    if (k >= P) return;
    const Split sp{G / P, G % P};
    const int64_t x0 = sp.start(k), x1 = sp.start(k + 1);
    // the pair holding x0 (binary search once; later segments move forward)
    int pi = 0;
    if constexpr (BATCH) {
        int lo = 0, hi = batch;  // prefix[lo] <= x0 < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= x0) lo = mid; else hi = mid;
        }
        pi = lo;
    }
    int64_t t = -1;
    Seg cur = make_seg<S, BATCH>(x0, x1, pi, t, a_data, a_off, b_data, b_off, c_data, c_off, n1, m1, prefix);
    int ci = 0, bi = 0, fold_ctr = 0;
    uint64_t acc[S];
    if (cur.jb1 - cur.jb0 > FIRST_CHUNK) {
        cur.f = FIRST_CHUNK;
        cur.nchunks = 1 + (cur.jb1 - cur.jb0 - FIRST_CHUNK + CHUNK_MAX - 1) / CHUNK_MAX;
    }
    stage_chunk<S, C::A_WORDS>(cur.a, cur.n, cur.b, cur.m, cur.d0, chunk_dims<KB>(cur.jb0, cur.jb1, 0, cur.f),
                               sm.buf, threadIdx.x, NTW);
    for (;;) {
        Seg nxt = cur;
        int nci = ci + 1;
        bool has_next = true;
        if (nci >= cur.nchunks) {
            if (cur.x_end < x1) {
                nxt = make_seg<S, BATCH>(cur.x_end, x1, pi, t, a_data, a_off, b_data, b_off, c_data, c_off,
                                         n1, m1, prefix);
                nci = 0;
            } else {
                has_next = false;
            }
        }
        if (has_next) {  // the next chunk streams in while this one is used
            stage_chunk<S, C::A_WORDS>(nxt.a, nxt.n, nxt.b, nxt.m, nxt.d0,
                                       chunk_dims<KB>(nxt.jb0, nxt.jb1, nci, nxt.f), sm.buf + (bi ^ 1) * C::BUF_WORDS,
                                       threadIdx.x, NTW);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (ci == 0) {
#pragma unroll
            for (int e = 0; e < S; ++e) acc[e] = 0;
            fold_ctr = 0;
        }
        const uint32_t* sA = sm.buf + bi * C::BUF_WORDS;
        compute_chunk<S, C::A_WORDS>(sA, sA + C::A_WORDS, chunk_dims<KB>(cur.jb0, cur.jb1, ci, cur.f).CL, mp, acc,
                                     fold_ctr, threadIdx.x >> 5, W);
        __syncthreads();  // this buffer is refilled by the next staging
        if (ci == cur.nchunks - 1) finish_segment<S, W>(cur, acc, mp, sm, sp, k, x0, sk, &s_last);
        if (!has_next) break;
        cur = nxt;
        ci = nci;
        bi ^= 1;
    }
}

// ---------------------------------------------------------------------------
// Warp-level form, for batches of small pairs.  The same positions and the
// same inner loop, but the unit of work belongs to a warp instead of a CTA,
// and warps claim units from a counter (one ahead of the unit they work on),
// so that warps the scheduler serves faster take more of them and the SMs
// finish together.  A unit is a whole pair when the pair has at most Q
// positions (all its tiles are then written directly), else one of the
// ceil(positions / Q) pieces of Q positions of the pair; only those pieces
// cut tiles, and a cut tile goes through the partial-sum slots of its pieces
// and the counter of its first piece as in the CTA form.  Units are claimed
// in three tiers, pieces first, then whole pairs of at least Q / 8 positions,
// then the rest, so that the last units handed out are small.  Q is set on the
// device from the total number of positions.  A warp stages its own chunks
// (double-buffered, WK_CHUNK coefficients of b) and keeps its own sums; no
// CTA-wide barrier remains.
// ---------------------------------------------------------------------------
constexpr int WK_WARPS = 8;           // independent warps per CTA
constexpr int WK_CHUNK = 256;         // b coefficients per warp chunk
constexpr int64_t WK_MIN_UNIT = 256;  // positions per piece, at least
constexpr int64_t WK_MAX_DEG = 4095;  // batches whose degrees stay below take this form
// pieces at most (two slots of TD words each per piece: 64 MiB for TD <= 256)
__host__ __device__ constexpr int64_t wk_units_max(int td) { return td <= 256 ? 32768 : 8 * 1024 * 1024 / td; }

// Schedule of the warp-level form, written by its planner.
struct WkPlan {
    int64_t* pos;        // [batch + 1] positions before pair i (as in the CTA form)
    int64_t* kbase;      // [batch + 1] pieces before pair i
    int64_t* rank;       // [batch] place of a whole pair within its tier (-1: the pair is cut in pieces)
    int64_t* bsum;       // [batch / 256] position sums of the count kernel's blocks
    int* unit_pair;      // [units] the pair of each unit, in claim order
    int64_t* sched;      // Q, units of tiers 0..2, claim counter
};

template <int S>
struct WCfg {
    static constexpr int TD = 32 * S;
    static constexpr int A_LOGICAL = FRONT + TD + WK_CHUNK + 8;
    static constexpr int A_CHUNKS = (A_LOGICAL + 3) / 4;
    static constexpr int A_WORDS = 4 * (A_CHUNKS + A_CHUNKS / 8 + 2);
    static constexpr int BUF_WORDS = A_WORDS + WK_CHUNK;
    static constexpr size_t SMEM = 4 * (size_t)WK_WARPS * 2 * BUF_WORDS;
};

// A warp's finished segment: its sums reduced mod p, then the tile's outputs
// or the piece's partial-sum slot.  Positions here are relative to the pair;
// piece v covers [v Q, v Q + Q) and the pair's pieces are numbered from kbase.
template <int S>
__device__ __forceinline__ void warp_finish(const Seg& sg, uint64_t (&acc)[S], const ModParams& mp, int64_t kbase,
                                            int64_t v, int64_t y0, int64_t Q, int64_t pbase, SkScratch sk) {
    constexpr int TD = 32 * S;
    const int lane = threadIdx.x & 31;
    const int L = sg.n + sg.m - 1;
    const int o0 = S * lane;
    uint32_t r[S];
#pragma unroll
    for (int e = 0; e < S; ++e) r[e] = barrett(fold2(acc[e], mp.c32), mp.p, mp.mu);
    if (sg.x == sg.s_tile && sg.x_end == sg.e_tile) {
#pragma unroll
        for (int e = 0; e < S; ++e)
            if (sg.d0 + o0 + e < L) sg.c[sg.d0 + o0 + e] = r[e];
        return;
    }
    // a cut tile (only pieces cut tiles): this piece's part goes to its slot (0
    // for the segment that starts the piece, 1 for the one that ends it); the
    // piece that arrives last at the counter of the tile's first piece adds
    // the parts, writes the outputs and resets the counter
    const int64_t ys = sg.s_tile - pbase, ye = sg.e_tile - pbase;
    const int64_t k1 = kbase + ys / Q, k2 = kbase + (ye - 1) / Q;
    // (the scratch holds 2 slots per piece, at most wk_units_max pieces, and their counters)
    if (!PM_CHK(k1 >= 0 && kbase + v < wk_units_max(TD) && k2 < wk_units_max(TD))) return;
    uint32_t* mine = sk.slots + (2 * (kbase + v) + (sg.x - pbase == y0 ? 0 : 1)) * TD;
#pragma unroll
    for (int e = 0; e < S; ++e) mine[o0 + e] = r[e];
    __syncwarp();
    int last = 0;
    if (lane == 0) {
        __threadfence();  // the warp's slot (ordered before by the warp barrier) before the count
        const unsigned int seen = atomicAdd(&sk.counters[k1], 1u);
        last = seen == (unsigned int)(k2 - k1) ? 1 : 0;
        if (last) __threadfence();
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    __syncwarp();
    if (last) {
        uint64_t sa[S], sb[S];
        const uint32_t* first = sk.slots + (2 * k1 + ((k1 - kbase) * Q == ys ? 0 : 1)) * TD + o0;
#pragma unroll
        for (int e = 0; e < S; ++e) { sa[e] = __ldcg(first + e); sb[e] = 0; }
        int64_t kk = k1 + 1;
        for (; kk + 1 <= k2; kk += 2) {  // two slots' reads in flight at a time
            const uint32_t* s0 = sk.slots + 2 * kk * TD + o0;
            const uint32_t* s1 = s0 + 2 * TD;
#pragma unroll
            for (int e = 0; e < S; ++e) { sa[e] += __ldcg(s0 + e); sb[e] += __ldcg(s1 + e); }
        }
        if (kk <= k2) {
#pragma unroll
            for (int e = 0; e < S; ++e) sa[e] += __ldcg(sk.slots + 2 * kk * TD + o0 + e);
        }
#pragma unroll
        for (int e = 0; e < S; ++e)
            if (sg.d0 + o0 + e < L) sg.c[sg.d0 + o0 + e] = barrett(sa[e] + sb[e], mp.p, mp.mu);
        if (lane == 0) sk.counters[k1] = 0;
    }
}

// Where a unit lies: pair i, its piece v (0 for a whole pair), the pair's
// first piece number kbase (pieces only) and its relative positions [y0, y1).
struct WkUnit {
    int i;
    int64_t v, kbase, y0, y1;
};

__device__ __forceinline__ WkUnit wk_decode(int64_t u, const WkPlan& pl, int64_t Q, int64_t tot0) {
    WkUnit w;
    w.i = pl.unit_pair[u];
    const int64_t npos = pl.pos[w.i + 1] - pl.pos[w.i];
    w.kbase = pl.kbase[w.i];
    const bool piece = u < tot0;
    w.v = piece ? u - w.kbase : 0;
    w.y0 = piece ? w.v * Q : 0;
    w.y1 = piece ? min(w.y0 + Q, npos) : npos;
    return w;
}

template <int S>
__global__ void __launch_bounds__(32 * WK_WARPS) plain_warp_kernel(
    const uint32_t* __restrict__ a_data, const int64_t* __restrict__ a_off,
    const uint32_t* __restrict__ b_data, const int64_t* __restrict__ b_off,
    uint32_t* __restrict__ c_data, const int64_t* __restrict__ c_off, int batch, WkPlan pl, ModParams mp,
    SkScratch sk) {
    using W = WCfg<S>;
    constexpr int KB = Cfg<S>::KB;
    extern __shared__ uint4 smem_raw[];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    uint32_t* buf = reinterpret_cast<uint32_t*>(smem_raw) + wi * 2 * W::BUF_WORDS;
    pdl_wait();  // the planner's schedule and unit table
    const int64_t Q = pl.sched[0];
    const int64_t tot0 = pl.sched[1];
    const int64_t U = tot0 + pl.sched[2] + pl.sched[3];
    unsigned long long* claim = reinterpret_cast<unsigned long long*>(pl.sched + 4);
    auto take = [&]() -> int64_t {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(claim, 1ull);
        return (int64_t)__shfl_sync(0xffffffffu, u, 0);
    };
    int64_t u = take();
    if (u >= U) return;  // (no CTA-wide barrier follows)
    int64_t u_next = take();  // claimed one ahead
    // the claim after that is issued at once and read at the next switch, so
    // that the atomic's round trip overlaps this unit's work
    unsigned long long pending = 0;
    if (lane == 0) pending = atomicAdd(claim, 1ull);
    WkUnit w = wk_decode(u, pl, Q, tot0);
    int pi = w.i;
    int64_t t = -1;
    Seg cur = make_seg<S, true, WK_CHUNK>(pl.pos[pi] + w.y0, pl.pos[pi] + w.y1, pi, t, a_data, a_off, b_data, b_off,
                                         c_data, c_off, 0, 0, pl.pos);
    int ci = 0, bi = 0, fold_ctr = 0;
    uint64_t acc[S];
    stage_chunk<S, W::A_WORDS, WK_CHUNK>(cur.a, cur.n, cur.b, cur.m, cur.d0,
                                         chunk_dims<KB, WK_CHUNK>(cur.jb0, cur.jb1, 0, cur.f), buf, lane, 32);
    for (;;) {
        // the chunk after this one: of this segment, of the unit's next segment, or of the next unit
        Seg nxt = cur;
        int nci = ci + 1;
        WkUnit nw = w;
        bool has_next = true, new_unit = false;
        if (nci >= cur.nchunks) {
            nci = 0;
            if (cur.x_end < pl.pos[w.i] + w.y1) {
                nxt = make_seg<S, true, WK_CHUNK>(cur.x_end, pl.pos[w.i] + w.y1, pi, t, a_data, a_off, b_data, b_off,
                                                  c_data, c_off, 0, 0, pl.pos);
            } else if (u_next < U) {
                nw = wk_decode(u_next, pl, Q, tot0);
                new_unit = true;
                pi = nw.i;
                t = -1;
                nxt = make_seg<S, true, WK_CHUNK>(pl.pos[pi] + nw.y0, pl.pos[pi] + nw.y1, pi, t, a_data, a_off,
                                                  b_data, b_off, c_data, c_off, 0, 0, pl.pos);
            } else {
                has_next = false;
            }
        }
        if (has_next) {
            stage_chunk<S, W::A_WORDS, WK_CHUNK>(nxt.a, nxt.n, nxt.b, nxt.m, nxt.d0,
                                                 chunk_dims<KB, WK_CHUNK>(nxt.jb0, nxt.jb1, nci, nxt.f),
                                                 buf + (bi ^ 1) * W::BUF_WORDS, lane, 32);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncwarp();
        if (ci == 0) {
#pragma unroll
            for (int e = 0; e < S; ++e) acc[e] = 0;
            fold_ctr = 0;
        }
        const uint32_t* sA = buf + bi * W::BUF_WORDS;
        compute_chunk<S, W::A_WORDS, WK_CHUNK>(sA, sA + W::A_WORDS, chunk_dims<KB, WK_CHUNK>(cur.jb0, cur.jb1, ci,
                                                                                             cur.f).CL,
                                               mp, acc, fold_ctr, 0, 1);
        __syncwarp();  // this buffer is refilled by the next staging
        if (ci == cur.nchunks - 1) warp_finish<S>(cur, acc, mp, w.kbase, w.v, w.y0, Q, pl.pos[w.i], sk);
        if (!has_next) break;
        if (new_unit) {  // moving to the claimed unit: the next claim is the pending one
            w = nw;
            u = u_next;
            u_next = (int64_t)__shfl_sync(0xffffffffu, pending, 0);
            if (lane == 0) pending = atomicAdd(claim, 1ull);
        }
        cur = nxt;
        ci = nci;
        bi ^= 1;
    }
}


// ---------------------------------------------------------------------------
// Batched form: a planner kernel validates the CSR layout and computes the
// position prefix over pairs; the persistent kernel above does the rest.
// Both are stream-ordered, so the pair can be captured in a CUDA graph.
// ---------------------------------------------------------------------------
constexpr int PLAN_THREADS = 1024;

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

__device__ __forceinline__ int64_t pair_positions(int64_t n, int64_t m, int64_t td) {
    if (n < m) { const int64_t t = n; n = m; m = t; }
    return cum_len(n, m, td, ntiles_of(n, m, td));
}

#ifndef PM_PLAIN_STUDY_TU
__global__ void __launch_bounds__(PLAN_THREADS) batch_plan_kernel(
    int batch, const int64_t* __restrict__ a_off, const int64_t* __restrict__ b_off,
    const int64_t* __restrict__ c_off, int64_t max_deg, int td, int64_t* prefix, int* status) {
    __shared__ long long s_scan[PLAN_THREADS];
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const int per = (batch + PLAN_THREADS - 1) / PLAN_THREADS;
    const int lo = min(batch, tid * per), hi = min(batch, lo + per);
    long long run = 0;
    for (int i = lo; i < hi; ++i) {
        int64_t n, m;
        if (!pair_dims(i, a_off, b_off, c_off, max_deg, &n, &m)) { s_bad = 1; continue; }
        run += pair_positions(n, m, td);
    }
    s_scan[tid] = run;
    __syncthreads();
    if (s_bad) {  // nothing is computed: G = 0
        for (int i = tid; i <= batch; i += PLAN_THREADS) prefix[i] = 0;
        if (tid == 0) atomicCAS(status, 0, (int)PM_ERR_INVALID_ARG);
        return;
    }
    for (int off = 1; off < PLAN_THREADS; off <<= 1) {
        const long long v = tid >= off ? s_scan[tid - off] : 0;
        __syncthreads();
        s_scan[tid] += v;
        __syncthreads();
    }
    long long pos = s_scan[tid] - run;
    for (int i = lo; i < hi; ++i) {
        int64_t n, m;
        pair_dims(i, a_off, b_off, c_off, max_deg, &n, &m);
        prefix[i] = pos;
        pos += pair_positions(n, m, td);
    }
    if (tid == PLAN_THREADS - 1) prefix[batch] = s_scan[PLAN_THREADS - 1];
}
#endif  // PM_PLAIN_STUDY_TU

// inclusive scan of one value per thread over the block
__device__ __forceinline__ long long block_scan(long long v, long long* sh) {
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int off = 1; off < PLAN_THREADS; off <<= 1) {
        const long long w = tid >= off ? sh[tid - off] : 0;
        __syncthreads();
        sh[tid] += w;
        __syncthreads();
    }
    const long long r = sh[tid];
    __syncthreads();
    return r;
}

// Planner of the warp-level form, in three kernels.  warp_count_kernel (one
// thread per pair): the pair's position count in pos[i] (-1 for a pair that
// fails the checks of batch_plan_kernel) and each block's sum in bsum.
// warp_plan_kernel (one CTA, only scans): Q from the total, the prefix of
// positions (in place), the pieces before each pair (kbase), each pair's place
// in the claim order (rank) and the three tiers' sizes.  warp_fill_kernel (one
// warp per pair): the table of the pair of every unit; it also resets the
// claim counter.
#ifndef PM_PLAIN_STUDY_TU
__global__ void __launch_bounds__(256) warp_count_kernel(int batch, const int64_t* __restrict__ a_off,
                                                         const int64_t* __restrict__ b_off,
                                                         const int64_t* __restrict__ c_off, int64_t max_deg, int td,
                                                         int64_t max_short, int64_t* __restrict__ pos,
                                                         int64_t* __restrict__ bsum) {
    __shared__ long long s_sum[8];
    pdl_trigger();  // the planner may be placed now; it waits for this kernel to end
    const int i = blockIdx.x * 256 + threadIdx.x;
    int64_t np = 0;
    if (i < batch) {
        int64_t n, m;
        // (a valid pair left to another form, min(n, m) >= max_short, counts no position)
        np = pair_dims(i, a_off, b_off, c_off, max_deg, &n, &m) ? (min(n, m) < max_short ? pair_positions(n, m, td) : 0)
                                                                : -1;
        pos[i] = np;
    }
    long long v = np > 0 ? np : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < 8; ++w) t += s_sum[w];
        bsum[blockIdx.x] = t;
    }
}
#endif  // PM_PLAIN_STUDY_TU

__device__ __forceinline__ int64_t div_up(int64_t x, int64_t q) {
    return (x < 0x7fffffff && q < 0x7fffffff) ? (int64_t)(((uint32_t)x + (uint32_t)q - 1) / (uint32_t)q)
                                               : (x + q - 1) / q;
}

// Inclusive scan over the block of three values per thread, by warp shuffles
// (two barriers); sh holds 3 x 32 words.
__device__ __forceinline__ void block_scan3(long long& x0, long long& x1, long long& x2, long long* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long y0 = __shfl_up_sync(0xffffffffu, x0, off);
        const long long y1 = __shfl_up_sync(0xffffffffu, x1, off);
        const long long y2 = __shfl_up_sync(0xffffffffu, x2, off);
        if (lane >= off) { x0 += y0; x1 += y1; x2 += y2; }
    }
    if (lane == 31) { sh[w] = x0; sh[32 + w] = x1; sh[64 + w] = x2; }
    __syncthreads();
    if (w == 0) {
        long long t0 = sh[lane], t1 = sh[32 + lane], t2 = sh[64 + lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long y0 = __shfl_up_sync(0xffffffffu, t0, off);
            const long long y1 = __shfl_up_sync(0xffffffffu, t1, off);
            const long long y2 = __shfl_up_sync(0xffffffffu, t2, off);
            if (lane >= off) { t0 += y0; t1 += y1; t2 += y2; }
        }
        sh[lane] = t0; sh[32 + lane] = t1; sh[64 + lane] = t2;
    }
    __syncthreads();
    if (w > 0) { x0 += sh[w - 1]; x1 += sh[32 + w - 1]; x2 += sh[64 + w - 1]; }
    __syncthreads();  // sh is free again
}

#ifndef PM_PLAIN_STUDY_TU
__global__ void __launch_bounds__(PLAN_THREADS) warp_plan_kernel(int batch, int td, int64_t q_min, WkPlan pl,
                                                                  int* status) {
    // pairs in rounds of PLAN_THREADS, pair r PLAN_THREADS + tid by thread tid
    __shared__ long long s_scan[96];
    __shared__ int s_bad;
    __shared__ long long s_round[4];
    pdl_wait();  // the count kernel's per-pair counts and block sums
    pdl_trigger();
    const int tid = threadIdx.x;
    const int rounds = (batch + PLAN_THREADS - 1) / PLAN_THREADS;
    __shared__ long long s_g;
    {
        long long t = 0;  // the count kernel's block sums
        for (int bidx = tid; bidx < (batch + 255) / 256; bidx += PLAN_THREADS) t += pl.bsum[bidx];
        long long d1 = 0, d2 = 0;
        block_scan3(t, d1, d2, s_scan);
        if (tid == PLAN_THREADS - 1) s_g = t;
        __syncthreads();
    }
    const int64_t G = s_g;
    const int64_t umax = wk_units_max(td);
    // pieces cut only pairs of more than Q positions: at most 2 G / Q of them
    const int64_t Q = max(q_min, (2 * G + umax - 1) / umax);
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // running totals of positions, pieces, tier-1 and tier-2 pairs
    long long bp = 0, b0 = 0, b1 = 0, b2 = 0;
    int64_t np_next = tid < batch ? pl.pos[tid] : 0;
    for (int r = 0; r < rounds; ++r) {
        const int i = r * PLAN_THREADS + tid;
        const int64_t np = np_next;
        // the next round's count is read now, its latency behind this round's scans
        // (this round overwrites only its own entries)
        np_next = i + PLAN_THREADS < batch ? pl.pos[i + PLAN_THREADS] : 0;
        if (np < 0) s_bad = 1;
        // (tier 3: no unit, for a pair past the batch, a bad pair, or one with no position)
        const int tier = (i >= batch || np <= 0) ? 3 : (np > Q ? 0 : (8 * np >= Q ? 1 : 2));
        const long long nu = tier == 0 ? div_up(np, Q) : 0;
        long long xp = np > 0 ? np : 0, x0 = nu, x1 = tier == 1;
        block_scan3(xp, x0, x1, s_scan);
        long long x2 = tier == 2, d1 = 0, d2 = 0;
        block_scan3(x2, d1, d2, s_scan);
        if (i < batch) {
            pl.pos[i] = bp + xp - (np > 0 ? np : 0);  // the count becomes the prefix
            pl.kbase[i] = b0 + x0 - nu;
            // rank: the tier-1 or tier-2 table slot (relative to the tier), -1 for pieces
            pl.rank[i] = tier == 1 ? b1 + x1 - 1 : (tier == 2 ? b2 + x2 - 1 : -1);
        }
        if (tid == PLAN_THREADS - 1) { s_round[0] = xp; s_round[1] = x0; s_round[2] = x1; s_round[3] = x2; }
        __syncthreads();
        bp += s_round[0];
        b0 += s_round[1];
        b1 += s_round[2];
        b2 += s_round[3];
        __syncthreads();
    }
    if (tid == 0) {
        const bool bad = s_bad != 0;
        if (bad) atomicCAS(status, 0, (int)PM_ERR_INVALID_ARG);
        pl.pos[batch] = G;
        pl.kbase[batch] = b0;
        pl.sched[0] = Q;
        pl.sched[1] = bad ? 0 : b0;  // nothing is computed for an invalid batch
        pl.sched[2] = bad ? 0 : b1;
        pl.sched[3] = bad ? 0 : b2;
    }
}
#endif  // PM_PLAIN_STUDY_TU

// The unit table (claim order: pieces, tier 1, tier 2), one warp per pair.
#ifndef PM_PLAIN_STUDY_TU
__global__ void __launch_bounds__(256) warp_fill_kernel(int batch, WkPlan pl) {
    pdl_wait();  // the plan kernel's schedule and ranks
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        pl.sched[4] = 0;  // claim counter
    }
    if (i >= batch) return;
    const int64_t tot0 = pl.sched[1], tot1 = pl.sched[2];
    const int64_t rk = pl.rank[i];
    if (rk >= 0) {
        if (lane == 0) {
            const int64_t np = pl.pos[i + 1] - pl.pos[i];
            const int64_t Q = pl.sched[0];
            pl.unit_pair[(8 * np >= Q ? tot0 : tot0 + tot1) + rk] = i;
        }
        return;
    }
    const int64_t k0 = pl.kbase[i], k1 = pl.kbase[i + 1];
    for (int64_t k = k0 + lane; k < k1; k += 32) pl.unit_pair[k] = i;
}
#endif  // PM_PLAIN_STUDY_TU

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------

// Raises the kernel's dynamic shared-memory limit and caches its occupancy,
// once per device (cache[dev] = blocks per SM, 0 = not yet set up).
template <typename K>
static cudaError_t kernel_setup(K kern, size_t smem, int dev, int* cache, int* occ,
                                int threads = NT) {
    if (dev >= 0 && dev < 64 && cache[dev] > 0) {
        *occ = cache[dev];
        return cudaSuccess;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int o = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, threads, smem);
    if (e != cudaSuccess) return e;
    o = std::max(o, 1);
    if (dev >= 0 && dev < 64) cache[dev] = o;
    *occ = o;
    return cudaSuccess;
}

// Scratch layout: COUNTER_REGION counters (zeroed when the buffer is allocated
// and returned to zero by every call), then 2 P slots of TD words.  Both forms
// keep their counters in this region (the CTA form one per CTA unit, at most
// COUNTER_MAX; the warp-level form one per piece, at most wk_units_max), so
// that a call of one form never finds the other's slots where it expects
// counters.
constexpr int64_t COUNTER_MAX = 4096;
constexpr int64_t COUNTER_REGION = COUNTER_REGION_DEV;
constexpr size_t COUNTER_BYTES = COUNTER_REGION * sizeof(unsigned int);
static_assert(wk_units_max(32) <= COUNTER_REGION && wk_units_max(256) <= COUNTER_REGION &&
                  wk_units_max(512) <= COUNTER_REGION && COUNTER_MAX <= COUNTER_REGION,
              "counters");

static size_t sk_bytes(int64_t P, int td) {
    return COUNTER_BYTES + (size_t)(2 * P * td) * sizeof(uint32_t);
}

static SkScratch sk_carve(void* base) {
    SkScratch s;
    s.counters = reinterpret_cast<unsigned int*>(base);
    s.slots = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(base) + COUNTER_BYTES);
    return s;
}

template <int S, int W = WB>
static pm_status launch_pair_s(const uint32_t* a, int n, const uint32_t* b, int m, uint32_t* c,
                               uint32_t p, cudaStream_t st, DeviceWorkspace* ws) {
    using C = Cfg<S, W>;
    auto kern = plain_sk_kernel<S, false, W>;
    static int occ_cache[64] = {};
    int occ = 0;
    cudaError_t e = kernel_setup(kern, C::SMEM, ws->device, occ_cache, &occ, 32 * W);
    if (e != cudaSuccess) return cuda_fail(e);
    const int64_t nn = std::max(n, m), mm = std::min(n, m);
    const int64_t G = cum_len(nn, mm, C::TD, ntiles_of(nn, mm, C::TD));
    const int64_t P = std::min<int64_t>(std::min<int64_t>((int64_t)ws->num_sms * occ, COUNTER_MAX),
                                        std::max<int64_t>(1, G / MIN_POSITIONS));
    StreamScratch* sc = nullptr;
    pm_status rc = stream_scratch(ws, st, &sc);
    if (rc != PM_OK) return rc;
    rc = ensure_scratch(&sc->sk, &sc->sk_bytes, sk_bytes(P, C::TD), st, /*zero=*/true);
    if (rc != PM_OK) return rc;
    const ModParams mp = host_mod_params(p, C::KB);
    e = chk_bind(ws);
    if (e != cudaSuccess) return cuda_fail(e);
    kern<<<(unsigned)P, 32 * W, C::SMEM, st>>>(a, nullptr, b, nullptr, c, nullptr, n, m, nullptr, 0, mp,
                                           sk_carve(sc->sk));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(1);
    return PM_OK;
}

#ifndef PM_PLAIN_STUDY_TU
pm_status launch_plain(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* c,
                       uint32_t p, int s, cudaStream_t st, DeviceWorkspace* ws) {
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
#endif  // PM_PLAIN_STUDY_TU

#ifndef PM_PLAIN_STUDY_TU
// Warp-level form of the batched product (degrees below WK_MAX_DEG).
template <int S>
static pm_status launch_batched_warp_s(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                                       const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                                       const int64_t* c_off, uint32_t p, int64_t max_deg, int64_t q_min,
                                       int64_t max_short, cudaStream_t st, DeviceWorkspace* ws) {
    using W = WCfg<S>;
    auto kern = plain_warp_kernel<S>;
    static int occ_cache[64] = {};
    int occ = 0;
    cudaError_t e = kernel_setup(kern, W::SMEM, ws->device, occ_cache, &occ, 32 * WK_WARPS);
    if (e != cudaSuccess) return cuda_fail(e);
    const int64_t grid = (int64_t)ws->num_sms * occ;
    StreamScratch* sc = nullptr;
    pm_status rc = stream_scratch(ws, st, &sc);
    if (rc != PM_OK) return rc;
    const int64_t umax = wk_units_max(W::TD);
    rc = ensure_scratch(&sc->sk, &sc->sk_bytes, sk_bytes(umax, W::TD), st, /*zero=*/true);
    if (rc != PM_OK) return rc;
    // sched (8), pos, kbase (batch + 1 each), rank (batch), block sums, unit table (umax + batch ints)
    const int64_t nblk = (batch + 255) / 256;
    rc = ensure_scratch(&sc->plan, &sc->plan_bytes,
                        sizeof(int64_t) * (size_t)(3 * batch + 2 + 8 + nblk) + sizeof(int) * (size_t)(umax + batch),
                        st, false);
    if (rc != PM_OK) return rc;
    const SkScratch sk = sk_carve(sc->sk);
    WkPlan pl;
    pl.sched = reinterpret_cast<int64_t*>(sc->plan);
    pl.pos = pl.sched + 8;
    pl.kbase = pl.pos + (batch + 1);
    pl.rank = pl.kbase + (batch + 1);
    pl.bsum = pl.rank + batch;
    pl.unit_pair = reinterpret_cast<int*>(pl.bsum + nblk);
    // three planning launches: the per-pair counts and the unit table are spread over many CTAs
    // (a one-CTA planner doing all three steps measured 12 us slower on 4096 pairs)
    const int64_t qm = q_min > 0 ? q_min : WK_MIN_UNIT;
    e = chk_bind(ws);
    if (e != cudaSuccess) return cuda_fail(e);
    warp_count_kernel<<<(unsigned)((batch + 255) / 256), 256, 0, st>>>((int)batch, a_off, b_off, c_off, max_deg,
                                                                      W::TD, max_short, pl.pos, pl.bsum);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_dep(warp_plan_kernel, dim3(1), dim3(PLAN_THREADS), 0, st, (int)batch, (int)W::TD, qm, pl,
                       ws->status);
    if (e == cudaSuccess)
        e = launch_dep(warp_fill_kernel, dim3((unsigned)((batch + 7) / 8)), dim3(256), 0, st, (int)batch, pl);
    if (e != cudaSuccess) return cuda_fail(e);
    const ModParams mp = host_mod_params(p, Cfg<S>::KB);
    e = launch_dep(kern, dim3((unsigned)grid), dim3(32 * WK_WARPS), (size_t)W::SMEM, st, a_data, a_off, b_data,
                   b_off, c_data, c_off, (int)batch, pl, mp, sk);
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(4);
    return PM_OK;
}


template <int S>
static pm_status launch_batched_s(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                                  const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                                  const int64_t* c_off, uint32_t p, int64_t max_deg, int64_t q_min,
                                  int64_t max_short, cudaStream_t st, DeviceWorkspace* ws) {
    if (max_deg <= WK_MAX_DEG && S <= 32)  // (64 sums per lane would spill in the warp form)
        return launch_batched_warp_s<S>(batch, a_data, a_off, b_data, b_off, c_data, c_off, p, max_deg, q_min,
                                        max_short, st, ws);
    if (max_short != PM_ALL_PAIRS) return PM_ERR_UNSUPPORTED;  // the CTA form computes every pair
    using C = Cfg<S>;
    auto kern = plain_sk_kernel<S, true>;
    static int occ_cache[64] = {};
    int occ = 0;
    cudaError_t e = kernel_setup(kern, C::SMEM, ws->device, occ_cache, &occ);
    if (e != cudaSuccess) return cuda_fail(e);
    const int64_t P = std::min<int64_t>((int64_t)ws->num_sms * occ, COUNTER_MAX);
    StreamScratch* sc = nullptr;
    pm_status rc = stream_scratch(ws, st, &sc);
    if (rc != PM_OK) return rc;
    rc = ensure_scratch(&sc->sk, &sc->sk_bytes, sk_bytes(P, C::TD), st, /*zero=*/true);
    if (rc != PM_OK) return rc;
    rc = ensure_scratch(&sc->plan, &sc->plan_bytes, sizeof(int64_t) * (size_t)(batch + 1), st, false);
    if (rc != PM_OK) return rc;
    int64_t* prefix = reinterpret_cast<int64_t*>(sc->plan);
    e = chk_bind(ws);
    if (e != cudaSuccess) return cuda_fail(e);
    batch_plan_kernel<<<1, PLAN_THREADS, 0, st>>>((int)batch, a_off, b_off, c_off, max_deg, C::TD,
                                                  prefix, ws->status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    const ModParams mp = host_mod_params(p, C::KB);
    kern<<<(unsigned)P, NT, C::SMEM, st>>>(a_data, a_off, b_data, b_off, c_data, c_off, 0, 0, prefix,
                                           (int)batch, mp, sk_carve(sc->sk));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(2);
    return PM_OK;
}

#endif  // PM_PLAIN_STUDY_TU
#ifndef PM_PLAIN_STUDY_TU
pm_status launch_batched_plain(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                               const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                               const int64_t* c_off, uint32_t p, int s, int64_t max_deg, int64_t q_min,
                               int64_t max_short, cudaStream_t st, DeviceWorkspace* ws) {
    switch (s) {
#define PM_CASE(SV) \
    case SV:        \
        return launch_batched_s<SV>(batch, a_data, a_off, b_data, b_off, c_data, c_off, p, max_deg, q_min, max_short, \
                                    st, ws);
        PM_CASE(1) PM_CASE(2) PM_CASE(4) PM_CASE(8) PM_CASE(16) PM_CASE(32) PM_CASE(64)
#undef PM_CASE
        default: return PM_ERR_INVALID_ARG;
    }
}
#endif  // PM_PLAIN_STUDY_TU

#ifdef PM_PLAIN_STUDY_TU
// The block-size study: the same product with l = 128, 256 or 512 threads per
// CTA (4, 8 or 16 warps; the paper's l of Section 5).
pm_status launch_plain_ell(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* c, uint32_t p,
                           int s, int ell, cudaStream_t st, DeviceWorkspace* ws) {
    const int ni = (int)n, mi = (int)m;
#define PM_ELL(W)                                                                   \
    switch (s) {                                                                    \
        case 1: return launch_pair_s<1, W>(a, ni, b, mi, c, p, st, ws);            \
        case 2: return launch_pair_s<2, W>(a, ni, b, mi, c, p, st, ws);            \
        case 4: return launch_pair_s<4, W>(a, ni, b, mi, c, p, st, ws);            \
        case 8: return launch_pair_s<8, W>(a, ni, b, mi, c, p, st, ws);            \
        case 16: return launch_pair_s<16, W>(a, ni, b, mi, c, p, st, ws);          \
        case 32: return launch_pair_s<32, W>(a, ni, b, mi, c, p, st, ws);          \
        case 64: return launch_pair_s<64, W>(a, ni, b, mi, c, p, st, ws);          \
        default: return PM_ERR_INVALID_ARG;                                         \
    }
    if (ell == 128) PM_ELL(4)
    if (ell == 512) PM_ELL(16)
    if (ell == 32 * WB) return launch_plain(a, n, b, m, c, p, s, st, ws);
#undef PM_ELL
    return PM_ERR_INVALID_ARG;
}
#endif  // PM_PLAIN_STUDY_TU

}  // namespace pm

#ifndef PM_PLAIN_STUDY_TU
// ---------------------------------------------------------------------------
// polymul_plain_noalloc: the single-pair product of polymul_plain with its
// scratch (partial-sum slots and tile counters) in a file-scope device array
// instead of library-allocated memory, for callers that cannot let a library
// call cudaMalloc (see include/polymul.h).  The kernel is plain_sk_kernel,
// unchanged; only where its scratch lives differs.
// ---------------------------------------------------------------------------
#include <mutex>

namespace pm {

constexpr size_t NOALLOC_BYTES = (size_t)4 << 20;  // per device that loads the library, held until exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[64] = {};  // device address of g_noalloc_scratch, per device

// Once per device, with that device current: the array's device address (the
// host-side symbol is only a stand-in) and cleared tile counters.
static pm_status noalloc_setup(int dev, cudaStream_t st, void** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_ptr[dev]) {
        *out = g_noalloc_ptr[dev];
        return PM_OK;
    }
    // the set-up's memset and device synchronisation would break a capture
    if (is_capturing(st)) return PM_ERR_UNSUPPORTED;
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMemset(ptr, 0, COUNTER_BYTES);  // the counters must start at zero
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e);
    g_noalloc_ptr[dev] = ptr;
    *out = ptr;
    return PM_OK;
}

template <int S>
static pm_status launch_pair_noalloc_s(const uint32_t* a, int n, const uint32_t* b, int m, uint32_t* c,
                                       uint32_t p, cudaStream_t st, int dev, int num_sms, void* scratch) {
    using C = Cfg<S>;
    auto kern = plain_sk_kernel<S, false>;
    static int occ_cache[64] = {};
    int occ = 0;
    cudaError_t e = kernel_setup(kern, C::SMEM, dev, occ_cache, &occ);
    if (e != cudaSuccess) return cuda_fail(e);
    const int64_t nn = std::max(n, m), mm = std::min(n, m);
    const int64_t G = cum_len(nn, mm, C::TD, ntiles_of(nn, mm, C::TD));
    const int64_t P = std::min<int64_t>(std::min<int64_t>((int64_t)num_sms * occ, COUNTER_MAX),
                                        std::max<int64_t>(1, G / MIN_POSITIONS));
    if (sk_bytes(P, C::TD) > NOALLOC_BYTES) return PM_ERR_RANGE;  // would not fit the static array
    const ModParams mp = host_mod_params(p, C::KB);
    kern<<<(unsigned)P, NT, C::SMEM, st>>>(a, nullptr, b, nullptr, c, nullptr, n, m, nullptr, 0, mp,
                                           sk_carve(scratch));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(1);
    return PM_OK;
}

}  // namespace pm

extern "C" pm_status polymul_plain_noalloc(const uint32_t* a, int64_t deg_a, const uint32_t* b,
                                           int64_t deg_b, uint32_t* c, uint32_t p, int s, void* stream) {
    using namespace pm;
    if (!a || !b || !c) return PM_ERR_INVALID_ARG;
    if (deg_a < 0 || deg_b < 0 || deg_a > PM_MAX_DEG || deg_b > PM_MAX_DEG) return PM_ERR_INVALID_ARG;
    if (p < 2 || p >= PM_MAX_P) return PM_ERR_RANGE;
    const int64_t L = deg_a + deg_b + 1;
    auto overlap = [](const void* x, int64_t xw, const void* y, int64_t yw) {
        const uintptr_t x0 = (uintptr_t)x, x1 = x0 + 4 * (uintptr_t)xw;
        const uintptr_t y0 = (uintptr_t)y, y1 = y0 + 4 * (uintptr_t)yw;
        return x0 < y1 && y0 < x1;
    };
    if (overlap(c, L, a, deg_a + 1) || overlap(c, L, b, deg_b + 1)) return PM_ERR_INVALID_ARG;
    if (s == 0) s = polymul_plain_default_s(deg_a, deg_b, p);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= 64) return PM_ERR_INTERNAL;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    cudaStream_t st = (cudaStream_t)stream;
    void* scratch = nullptr;
    pm_status rc = noalloc_setup(dev, st, &scratch);
    if (rc != PM_OK) return rc;
    const uint32_t *x = a, *y = b;
    int n = (int)(deg_a + 1), m = (int)(deg_b + 1);
    switch (s) {
        case 1: return launch_pair_noalloc_s<1>(x, n, y, m, c, p, st, dev, sms, scratch);
        case 2: return launch_pair_noalloc_s<2>(x, n, y, m, c, p, st, dev, sms, scratch);
        case 4: return launch_pair_noalloc_s<4>(x, n, y, m, c, p, st, dev, sms, scratch);
        case 8: return launch_pair_noalloc_s<8>(x, n, y, m, c, p, st, dev, sms, scratch);
        case 16: return launch_pair_noalloc_s<16>(x, n, y, m, c, p, st, dev, sms, scratch);
        case 32: return launch_pair_noalloc_s<32>(x, n, y, m, c, p, st, dev, sms, scratch);
        case 64: return launch_pair_noalloc_s<64>(x, n, y, m, c, p, st, dev, sms, scratch);
        default: return PM_ERR_INVALID_ARG;
    }
}

#endif  // PM_PLAIN_STUDY_TU