// Tensor-core form of the batched product (tcgen05, bf16 limbs, fp32 accumulation).
//
// The paper has no tensor-core path; this computes the same residues as the
// long multiplication of Section 5 by turning each product into a sum of
// exact small-integer matrix products.
//
// Limbs.  Coefficients are first moved to the centred range (-p/2, p/2]
// (same residue).  b is split into 4 balanced base-256 digits d_j in
// [-128, 127], a into 5 balanced base-64 digits e_i in [-32, 31]; bf16 holds
// both exactly.  Then
//     c = sum_{i<5, j<4} 64^i 256^j (e_i * d_j)   (mod p),
// and every entry of a digit convolution e_i * d_j is a sum of at most
// min(n, m) <= 4096 products of magnitude <= 128 * 32 = 2^12, so it stays
// within 2^24 in magnitude and the tensor core's fp32 accumulation is exact.
// (tcgen05 kind::i8 would hold larger limbs, but ptxas rejects it for
// sm_103a.)
//
// Matrix form (T = 32 outputs per block, block I covers outputs 32 I .. 32 I + 31;
// the K index runs backwards, k' = 31 - k, in both operands):
//     D[(j, r)][(I, i)] = sum_delta sum_{k'<32} d_j[32 delta - 31 + r + k'] * e_i[32 (I - delta) + 31 - k']
//                       = (e_i * d_j)[32 I + r].
// For one shift delta this is one 128 x 240 x 32 product (two MMAs of K = 16):
// N = 240 columns are 48 output blocks times the 5 limbs of a; the a operand
// is stored once per tile as rows (J, i) = limb i of block J of a, reversed,
// and the rows shift delta needs are the same rows moved by 5 per delta, so
// its descriptor just starts 5 * 16 bytes earlier for each delta.  M = 128
// rows are the 4 limbs of b times 32 offsets r, ordered (r / 8, limb j, r mod 8)
// so that one descriptor covers all limbs: with k' reversed, the 8 x 8 core
// matrix of limb j at row group r / 8 = g and K chunk c holds
// d_j[32 delta - 31 + 8 (g + c) + row + column], a Hankel block that depends
// only on q = 4 delta + g + c.  These core matrices H_j[q] are built once per
// q in shared memory, the 4 limbs interleaved (512 bytes per q), and the
// descriptor walks them with 128 bytes between row groups (the next limb or,
// after 4 limbs, the next g) and 512 bytes between K chunks (the next q).  A
// shift thus costs 4 new core matrices per limb instead of a 128 x 32 block.
// All shifts accumulate into one TMEM tile (240 fp32 columns x 128 lanes).
//
// Epilogue.  TMEM lane 32 g + 8 j + t holds D[(j, 8 g + t)][.]: warp g reads
// its 32 lanes, each thread forms sum_i 64^i D (exact in int64), reduces it
// mod p and multiplies by 256^j mod p, and the 4 limbs of one output are
// added with two warp shuffles before the store.
//
// Work: tiles of 1536 outputs of every pair, taken by persistent CTAs (one
// per SM) from an atomic counter.  Every wait on an mbarrier is bounded: when
// it runs out the kernel records PM_ERR_TIMEOUT and skips the remaining work.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace pm {

constexpr int TT = 32;                     // outputs per block
constexpr int NBLK = 48;                   // blocks per tile
constexpr int NA_LIMB = 5, NB_LIMB = 4;
constexpr int MMA_M = 128, MMA_N = NBLK * NA_LIMB;  // 240
constexpr int TILE_OUT = TT * NBLK;        // 1536
constexpr int TC_MAXK = 4096;              // exactness bound on min(n, m)
constexpr int TC_THREADS = 256;
constexpr int GROUP_D = 8;                 // shifts per A-operand group (two groups in flight)
constexpr int MAX_DELTA = TC_MAXK / TT + 2;            // shifts a tile can need
constexpr int BD_SHIFT = 7;                            // staged b digit t sits at index t + 7
constexpr int BD_LEN = TT * (MAX_DELTA + 2);           // b digits staged per limb (with the shift)
constexpr int ROWS_MAX = NA_LIMB * (NBLK + MAX_DELTA + 2);
constexpr int B_LBO = ROWS_MAX * 16;                   // bytes between K chunks of the a operand
constexpr int H_Q = 4 * GROUP_D + 4;                  // Hankel core-matrix indices per group (4 G + 3 used)
constexpr int H_SLOT = H_Q * 512;                      // 4 limbs x 128-byte core matrices per index
constexpr uint32_t TMEM_COLS = 256;
constexpr int64_t WAIT_LIMIT = 1ll << 26;              // polls before a wait is declared lost

// shared memory map (bytes)
constexpr int SM_B = 0;                                   // a operand: 4 chunks x ROWS_MAX rows
constexpr int SM_H = SM_B + 4 * B_LBO;                    // 2 groups of Hankel core matrices
constexpr int SM_BD = SM_H + 2 * H_SLOT;                  // b digits: NB_LIMB x BD_LEN bf16
constexpr int RAW_A = TT * (NBLK + MAX_DELTA);            // raw coefficients of a per tile
constexpr int RAW_B = BD_LEN;                             // raw coefficients of b per tile
constexpr int SM_RAW = SM_BD + NB_LIMB * BD_LEN * 2;      // the next tile's raw coefficients
constexpr int SM_CTL = SM_RAW + 4 * (RAW_A + RAW_B);      // mbarriers, TMEM address, tile id
constexpr int TC_SMEM = SM_CTL + 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, K-major, no swizzle: core matrices
// of 8 rows x 16 bytes; lbo = bytes between K-adjacent core matrices, sbo =
// bytes between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of sm_100 family
    return d;
}

// instruction descriptor: D f32, A and B bf16, both K-major, N and M as given
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(MMA_N >> 3) << 17) |
                           ((uint32_t)(MMA_M >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false if it ran out.
__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity) {
    for (int64_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ uint16_t bf16_bits(int v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn((float)v));  // exact for |v| <= 256
}

// balanced digits of the centred representative of x in [0, p)
__device__ __forceinline__ int centred(uint32_t x, uint32_t p) {
    return x > (p - 1) / 2 ? (int)x - (int)p : (int)x;
}

// Geometry of one tile (see the kernel): pair, shifts, staged blocks.
struct TcTile {
    const uint32_t* a;
    const uint32_t* b;
    uint32_t* c;
    int n, m, L, I0, d_lo, d_hi, nd, J_min, nJ, tb0;
};

__device__ __forceinline__ TcTile make_tile(int64_t tile, int batch, const uint32_t* __restrict__ a_data,
                                            const int64_t* __restrict__ a_off, const uint32_t* __restrict__ b_data,
                                            const int64_t* __restrict__ b_off, uint32_t* __restrict__ c_data,
                                            const int64_t* __restrict__ c_off, const int64_t* __restrict__ prefix) {
    TcTile tt;
    int lo = 0, hi = batch;  // the pair: prefix[lo] <= tile < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= tile) lo = mid; else hi = mid;
    }
    tt.a = a_data + a_off[lo];
    tt.b = b_data + b_off[lo];
    tt.c = c_data + c_off[lo];
    tt.n = (int)(a_off[lo + 1] - a_off[lo]);
    tt.m = (int)(b_off[lo + 1] - b_off[lo]);
    if (tt.m > tt.n) {  // b is the shorter operand (fewer shifts per tile)
        const uint32_t* t = tt.a; tt.a = tt.b; tt.b = t;
        const int tn = tt.n; tt.n = tt.m; tt.m = tn;
    }
    tt.L = tt.n + tt.m - 1;
    tt.I0 = (int)(tile - prefix[lo]) * NBLK;           // first output block of the tile
    const int NA = (tt.n + TT - 1) / TT;                // blocks of a
    const int dmax = (tt.m + TT - 2) / TT;              // largest shift meeting b
    tt.d_lo = max(0, tt.I0 - NA + 1);
    tt.d_hi = min(dmax, tt.I0 + NBLK - 1);
    tt.nd = tt.d_hi - tt.d_lo + 1;                      // >= 1 for a tile inside [0, L)
    tt.J_min = tt.I0 - tt.d_hi;
    tt.nJ = NBLK + tt.d_hi - tt.d_lo;                   // blocks J_min .. J_min + nJ - 1
    tt.tb0 = TT * tt.d_lo - TT;                         // first staged b index
    return tt;
}

// 4-byte asynchronous copy; with valid == false it writes a zero and reads nothing.
__device__ __forceinline__ void cp_async4_tc(uint32_t* dst, const uint32_t* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

// Starts the copies of a tile's raw coefficients: a[32 J_min ..] (nJ blocks)
// and b[tb0 ..] (32 (nd + 2) words), zeros outside the operands.
__device__ __forceinline__ void prefetch_raw(const TcTile& tt, uint32_t* rawA, uint32_t* rawB) {
    for (int q = threadIdx.x; q < tt.nJ * TT; q += blockDim.x) {
        const int g = tt.J_min * TT + q;
        const bool v = g >= 0 && g < tt.n;
        cp_async4_tc(rawA + q, tt.a + (v ? g : 0), v);
    }
    for (int t = threadIdx.x; t < TT * (tt.nd + 2); t += blockDim.x) {
        const int g = tt.tb0 + t;
        const bool v = g >= 0 && g < tt.m;
        cp_async4_tc(rawB + t, tt.b + (v ? g : 0), v);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

struct TcParams {
    uint32_t p;
    uint64_t mu;          // floor(2^64 / p)
    uint64_t off;         // a multiple of p above 2^52 (makes signed limb sums non-negative)
    uint32_t w256[NB_LIMB];  // 256^j mod p
};

__global__ void __launch_bounds__(TC_THREADS, 1) tc_batched_kernel(
    int batch, const uint32_t* __restrict__ a_data, const int64_t* __restrict__ a_off,
    const uint32_t* __restrict__ b_data, const int64_t* __restrict__ b_off,
    uint32_t* __restrict__ c_data, const int64_t* __restrict__ c_off, const int64_t* __restrict__ prefix,
    unsigned int* __restrict__ counter, TcParams tp, int* status) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t* sB = sm + SM_B;
    uint8_t* sH = sm + SM_H;
    uint16_t* sbd = reinterpret_cast<uint16_t*>(sm + SM_BD);
    uint32_t* rawA = reinterpret_cast<uint32_t*>(sm + SM_RAW);
    uint32_t* rawB = rawA + RAW_A;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + SM_CTL);  // 2 mbarriers
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + SM_CTL + 32);
    int* s_tile = reinterpret_cast<int*>(sm + SM_CTL + 48);
    int* s_abort = reinterpret_cast<int*>(sm + SM_CTL + 52);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar0 = smem_u32(bars), bar1 = smem_u32(bars + 1);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar1), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    uint32_t parity[2] = {0, 0};
    const int64_t total = prefix[batch];

    if (tid == 0) *s_tile = (int)atomicAdd(counter, 1u);
    __syncthreads();
    int64_t tile = *s_tile;
    TcTile cur{};
    if (tile < total) {
        cur = make_tile(tile, batch, a_data, a_off, b_data, b_off, c_data, c_off, prefix);
        prefetch_raw(cur, rawA, rawB);
    }
    for (;;) {
        if (tile >= total || *s_abort) break;
        uint32_t* c = cur.c;
        const int L = cur.L, I0 = cur.I0;
        const int d_lo = cur.d_lo, d_hi = cur.d_hi, nd = cur.nd, nJ = cur.nJ, tb0 = cur.tb0;
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();

        // ---- digits of the staged coefficients: b (natural order) and the a operand ----
        for (int t = tid; t < TT * (nd + 2); t += TC_THREADS) {
            int v = centred(rawB[t], tp.p);
#pragma unroll
            for (int j = 0; j < NB_LIMB; ++j) {
                const int d = ((v + 128) & 255) - 128;
                sbd[j * BD_LEN + BD_SHIFT + t] = bf16_bits(d);  // shifted: core matrices start 16-byte aligned
                v = (v - d) >> 8;
            }
        }
        for (int q = tid; q < nJ * TT; q += TC_THREADS) {
            const int Jr = q / TT, k = q % TT;
            int v = centred(rawA[q], tp.p);
#pragma unroll
            for (int i = 0; i < NA_LIMB; ++i) {
                const int d = ((v + 32) & 63) - 32;
                const int row = NA_LIMB * Jr + i, kr = TT - 1 - k;  // K runs backwards
                *reinterpret_cast<uint16_t*>(sB + (kr >> 3) * B_LBO + row * 16 + (kr & 7) * 2) = bf16_bits(d);
                v = (v - d) >> 6;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // claim the next tile; its coefficients stream in while this tile's products run
        if (tid == 0) *s_tile = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int64_t next = *s_tile;
        TcTile nxt{};
        if (next < total) {
            nxt = make_tile(next, batch, a_data, a_off, b_data, b_off, c_data, c_off, prefix);
            prefetch_raw(nxt, rawA, rawB);
        }

        // ---- shifts in groups of GROUP_D: build the Toeplitz blocks, issue the MMAs ----
        const int ngroups = (nd + GROUP_D - 1) / GROUP_D;
        for (int gi = 0; gi < ngroups && !*s_abort; ++gi) {
            const int buf = gi & 1;
            if (gi >= 2) {
                if (!wait_parity(buf ? bar1 : bar0, parity[buf])) {
                    atomicCAS(status, 0, (int)PM_ERR_TIMEOUT);
                    *s_abort = 1;
                }
                parity[buf] ^= 1u;
            }
            __syncthreads();
            if (*s_abort) break;
            uint8_t* hslot = sH + buf * H_SLOT;
            const int nds = min(GROUP_D, nd - gi * GROUP_D);
            const int dg = d_lo + gi * GROUP_D;  // first shift of the group
            // core matrix H_j[q] (q = 4 dg + qq): row t holds d_j[-31 + 8 q + t .. + 7], 8 ascending
            // digits; its 8 rows are the 16 digits from d_j[-31 + 8 q] shifted by 0..7
            for (int w = tid; w < (4 * nds + 3) * NB_LIMB; w += TC_THREADS) {
                const int qq = w >> 2, j = w & 3;
                // staged index of d_j[-31 + 8 q] plus BD_SHIFT: a multiple of 8
                const int i0 = BD_SHIFT - 31 + 8 * (4 * dg + qq) - tb0;
                const uint4 lo4 = *reinterpret_cast<const uint4*>(sbd + j * BD_LEN + i0);
                const uint4 hi4 = *reinterpret_cast<const uint4*>(sbd + j * BD_LEN + i0 + 8);
                const uint32_t wd[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
                uint8_t* dst = hslot + qq * 512 + j * 128;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int k = t >> 1;
                    uint4 v;
                    if ((t & 1) == 0) {
                        v = make_uint4(wd[k], wd[k + 1], wd[k + 2], wd[k + 3]);
                    } else {
                        v = make_uint4(__funnelshift_r(wd[k], wd[k + 1], 16), __funnelshift_r(wd[k + 1], wd[k + 2], 16),
                                       __funnelshift_r(wd[k + 2], wd[k + 3], 16), __funnelshift_r(wd[k + 3], wd[k + 4], 16));
                    }
                    *reinterpret_cast<uint4*>(dst + t * 16) = v;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int s = 0; s < nds; ++s) {
                    const int d = dg + s;
                    const uint32_t b_addr = smem_u32(sB) + (uint32_t)(NA_LIMB * (d_hi - d) * 16);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint64_t da = smem_desc(smem_u32(hslot) + (uint32_t)((4 * s + 2 * h) * 512), 512, 128);
                        const uint64_t db = smem_desc(b_addr + 2 * h * B_LBO, B_LBO, 128);
                        mma_bf16(tmem, da, db, (gi == 0 && s == 0 && h == 0) ? 0u : 1u);
                    }
                }
                mma_commit(buf ? bar1 : bar0);
            }
        }
        // ---- wait for the outstanding groups (in issue order) ----
        for (int gi = max(0, ngroups - 2); gi < ngroups; ++gi) {
            const int buf = gi & 1;
            if (!*s_abort && !wait_parity(buf ? bar1 : bar0, parity[buf])) {
                atomicCAS(status, 0, (int)PM_ERR_TIMEOUT);
                *s_abort = 1;
            }
            parity[buf] ^= 1u;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (*s_abort) break;

        // ---- epilogue: warp g reads TMEM lanes 32 g .. 32 g + 31 = (limb j, offset 8 g + t) ----
        if (warp < 4) {
            const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
            const int j = lane >> 3, r = 8 * warp + (lane & 7);
            const uint64_t wj = tp.w256[j];
            for (int c0 = 0; c0 < MMA_N; c0 += 80) {  // 16 blocks x 5 limbs per round
                uint32_t rr[80];
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(rr[16 * q + 0]), "=r"(rr[16 * q + 1]), "=r"(rr[16 * q + 2]), "=r"(rr[16 * q + 3]),
                          "=r"(rr[16 * q + 4]), "=r"(rr[16 * q + 5]), "=r"(rr[16 * q + 6]), "=r"(rr[16 * q + 7]),
                          "=r"(rr[16 * q + 8]), "=r"(rr[16 * q + 9]), "=r"(rr[16 * q + 10]), "=r"(rr[16 * q + 11]),
                          "=r"(rr[16 * q + 12]), "=r"(rr[16 * q + 13]), "=r"(rr[16 * q + 14]), "=r"(rr[16 * q + 15])
                        : "r"(tmem + lane_base + (uint32_t)(c0 + 16 * q)));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int ib = 0; ib < 16; ++ib) {
                    int64_t sum = 0;
#pragma unroll
                    for (int i = NA_LIMB - 1; i >= 0; --i)
                        sum = sum * 64 + (int64_t)__float2int_rn(__uint_as_float(rr[NA_LIMB * ib + i]));
                    const uint32_t v = barrett((uint64_t)(sum + (int64_t)tp.off), tp.p, tp.mu);
                    uint32_t x = barrett((uint64_t)v * wj, tp.p, tp.mu);
                    x += __shfl_xor_sync(0xffffffffu, x, 8);   // limbs j and j^1
                    x = barrett((uint64_t)x, tp.p, tp.mu);
                    x += __shfl_xor_sync(0xffffffffu, x, 16);  // and j^2
                    const int g = (I0 + c0 / NA_LIMB + ib) * TT + r;
                    if (j == 0 && g < L) c[g] = barrett((uint64_t)x, tp.p, tp.mu);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        cur = nxt;
        tile = next;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // no copy outlives the CTA
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// Planner: validates the CSR layout (degrees <= max_deg <= 4095) and builds
// the prefix of tile counts; resets the tile counter.
__global__ void __launch_bounds__(1024) tc_plan_kernel(int batch, const int64_t* __restrict__ a_off,
                                                        const int64_t* __restrict__ b_off,
                                                        const int64_t* __restrict__ c_off, int64_t max_deg,
                                                        int64_t* prefix, unsigned int* counter, int* status) {
    __shared__ long long s_scan[1024];
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const int per = (batch + 1023) / 1024;
    const int lo = min(batch, tid * per), hi = min(batch, lo + per);
    long long run = 0;
    for (int i = lo; i < hi; ++i) {
        const int64_t n = a_off[i + 1] - a_off[i], m = b_off[i + 1] - b_off[i], l = c_off[i + 1] - c_off[i];
        if (n < 1 || m < 1 || n - 1 > max_deg || m - 1 > max_deg || l != n + m - 1 || a_off[i] < 0 ||
            b_off[i] < 0 || c_off[i] < 0) {
            s_bad = 1;
            continue;
        }
        run += (n + m - 1 + TILE_OUT - 1) / TILE_OUT;
    }
    s_scan[tid] = run;
    __syncthreads();
    if (s_bad) {
        for (int i = tid; i <= batch; i += 1024) prefix[i] = 0;
        if (tid == 0) {
            atomicCAS(status, 0, (int)PM_ERR_INVALID_ARG);
            *counter = 0;
        }
        return;
    }
    for (int off = 1; off < 1024; off <<= 1) {
        const long long v = tid >= off ? s_scan[tid - off] : 0;
        __syncthreads();
        s_scan[tid] += v;
        __syncthreads();
    }
    long long pos = s_scan[tid] - run;
    for (int i = lo; i < hi; ++i) {
        prefix[i] = pos;
        const int64_t n = a_off[i + 1] - a_off[i], m = b_off[i + 1] - b_off[i];
        pos += (n + m - 1 + TILE_OUT - 1) / TILE_OUT;
    }
    if (tid == 1023) {
        prefix[batch] = s_scan[1023];
        *counter = 0;
    }
}

pm_status launch_batched_tensor(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                                const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                                const int64_t* c_off, uint32_t p, int64_t max_deg, cudaStream_t st,
                                DeviceWorkspace* ws) {
    if (p >= (1u << 29) || max_deg + 1 > TC_MAXK) return PM_ERR_UNSUPPORTED;
    if (ws->cc_major != 10) return PM_ERR_UNSUPPORTED;  // tcgen05 needs the sm_100 family
    StreamScratch* sc = nullptr;
    pm_status rc = stream_scratch(ws, st, &sc);
    if (rc != PM_OK) return rc;
    rc = ensure_scratch(&sc->tc, &sc->tc_bytes, 256 + sizeof(int64_t) * (size_t)(batch + 1), st, false);
    if (rc != PM_OK) return rc;
    unsigned int* counter = reinterpret_cast<unsigned int*>(sc->tc);
    int64_t* prefix = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(sc->tc) + 256);
    static int done[64] = {};
    cudaError_t e;
    if (!done[ws->device]) {
        e = cudaFuncSetAttribute(tc_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        if (e != cudaSuccess) return cuda_fail(e);
        done[ws->device] = 1;
    }
    TcParams tp;
    tp.p = p;
    tp.mu = (uint64_t)(((unsigned __int128)1 << 64) / p);
    tp.off = ((1ull << 52) / p + 1) * (uint64_t)p;
    uint64_t w = 1;
    for (int j = 0; j < NB_LIMB; ++j) {
        tp.w256[j] = (uint32_t)w;
        w = (w * 256) % p;
    }
    tc_plan_kernel<<<1, 1024, 0, st>>>((int)batch, a_off, b_off, c_off, max_deg, prefix, counter, ws->status);
    tc_batched_kernel<<<ws->num_sms, TC_THREADS, TC_SMEM, st>>>((int)batch, a_data, a_off, b_data, b_off,
                                                                c_data, c_off, prefix, counter, tp, ws->status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(2);
    return PM_OK;
}

}  // namespace pm
