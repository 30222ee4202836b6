// Number-theoretic-transform form of the product (large degrees).
//
// c = a*b mod p as the inverse transform of the pointwise product of the
// length-N transforms of a and b (N = 2^k >= n+m-1, N | p-1), scaled by N^-1.
// The paper has no transform path; the result is the same exact residues as
// the long multiplication of Section 5.
//
// Layout of a length-N transform, N = N1 * N2 with N2 = 4096 when N > 4096
// (four-step decomposition; n = n1 N2 + n2, k = k1 + N1 k2):
//   X[k1 + N1 k2] = sum_n2 w_N2^(n2 k2) w_N^(n2 k1) sum_n1 x[n1 N2 + n2] w_N1^(n1 k1)
// 1. column pass: for each column n2 a length-N1 transform over n1, times
//    w_N^(n2 k1); a and b in one launch, written to two scratch arrays;
// 2. row pass (fused): per row, the length-N2 transforms of both arrays, the
//    pointwise product, the inverse length-N2 transform and w_N^(-n2 k1);
// 3. inverse column pass: per column the inverse length-N1 transform, the
//    scale N^-1, and the store of the n+m-1 output words.
// Every pass reads and writes each word once (3 HBM round trips in all).
// Forward transforms are decimation in frequency (natural order in,
// digit-reversed out), inverse ones decimation in time (digit-reversed in,
// natural out), with radix-4 butterflies and one radix-2 stage when log2 of
// the length is odd, so no reordering pass is needed.  The column transforms
// run level by level in shared memory, 8 or 16 adjacent columns per CTA; the
// length-4096 row transforms run as three radix-16 stages in registers (16
// elements per thread, two radix-4 levels per stage) with two shared-memory
// exchanges, and the pointwise product sits between the last forward and the
// first inverse stage without leaving registers.  N <= 4096 runs in one CTA
// per product: from 1024 points on, the row pass's length-4096 transform on a
// and b zero-padded to 4096 words; below that (and for primes whose 2-adic
// order is below 12) length-N transforms level by level in shared memory.
//
// Arithmetic: the four-step passes and the one-CTA row transform keep values
// in [0, 2p) between butterflies (the lazy forms below; 4p < 2^32 since
// p < 2^30) and the final scale makes them canonical; the level-by-level
// shared-memory path keeps them in [0, p).
// Multiplication by a table
// constant w uses Shoup's precomputed quotient wq = floor(w 2^32 / p)
// (V. Shoup, NTL; also D. Harvey, "Faster arithmetic for number-theoretic
// transforms", J. Symb. Comp. 2014): q = hi32(x wq), r = x w - q p in [0, 2p).
// The pointwise product uses Montgomery reduction (P. Montgomery,
// "Modular multiplication without trial division", Math. Comp. 1985) with
// R = 2^32; the extra factor 2^-32 is folded into the final scale
// N^-1 2^32 mod p.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace pm {

constexpr int NTT_N2_LOG = 12;               // row length of the four-step layout
constexpr int NTT_N2 = 1 << NTT_N2_LOG;
constexpr int NTT_MAX_LOG = 24;              // N1 <= 4096 keeps a column block in shared memory
constexpr int NTT_THREADS = 512;
#ifndef NTT_ROW_MINB
#define NTT_ROW_MINB 3   // row-pass CTAs per SM the compiler must fit (80 registers, no spills)
#endif
#ifndef NTT_COL_MINB
#define NTT_COL_MINB 2   // column-pass CTAs per SM the compiler must fit (3 would cap at 40 registers and spill)
#endif
#ifndef NTT_COLS8_LOG
#define NTT_COLS8_LOG 11 // column blocks of 8 (not 16) from this log2 N1 on: 64 KiB per CTA, 3 CTAs per SM
#endif

struct NttMod {
    uint32_t p;
    uint32_t pinv_neg;  // -p^-1 mod 2^32
};

__device__ __forceinline__ uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint32_t add_p(uint32_t x, uint32_t y, uint32_t p) {
    const uint32_t s = x + y;
    return umin32(s, s - p);
}
__device__ __forceinline__ uint32_t sub_p(uint32_t x, uint32_t y, uint32_t p) {
    const uint32_t d = x - y + p;
    return umin32(d, d - p);
}
__device__ __forceinline__ uint32_t mul_shoup(uint32_t x, uint2 w, uint32_t p) {
    const uint32_t q = __umulhi(x, w.y);
    const uint32_t r = x * w.x - q * p;
    return umin32(r, r - p);
}
__device__ __forceinline__ uint32_t mul_mont(uint32_t x, uint32_t y, const NttMod& m) {
    const uint64_t t = (uint64_t)x * y;
    const uint32_t q = (uint32_t)t * m.pinv_neg;
    const uint32_t u = (uint32_t)((t + (uint64_t)q * m.p) >> 32);
    return umin32(u, u - m.p);
}

// Lazy forms (D. Harvey, "Faster arithmetic for number-theoretic transforms",
// J. Symb. Comp. 2014) for the four-step passes: values stay in [0, 2p)
// between butterflies and only the final scale makes them canonical.
// Shoup's product without its correction: for any x < 2^32, r in [0, 2p).
__device__ __forceinline__ uint32_t mul_shoup_lz(uint32_t x, uint2 w, uint32_t p) {
    return x * w.x - __umulhi(x, w.y) * p;
}
// v < 4p to [0, 2p) (p2 = 2p)
__device__ __forceinline__ uint32_t r2p(uint32_t v, uint32_t p2) { return umin32(v, v - p2); }
// Montgomery's product of x, y < 2p without its correction: (x y + q p) / 2^32 < 2p
// since 4p < 2^32.
__device__ __forceinline__ uint32_t mul_mont_lz(uint32_t x, uint32_t y, const NttMod& m) {
    const uint64_t t = (uint64_t)x * y;
    const uint32_t q = (uint32_t)t * m.pinv_neg;
    return (uint32_t)((t + (uint64_t)q * m.p) >> 32);
}

// Frequency index k of output position `pos` of a forward transform of
// length 2^logm (stage radices 2 (odd logm only) then 4, 4, ...): the base-4
// digits of the position, read in reverse (after the leading binary digit
// when logm is odd, which becomes the lowest digit of k).
__host__ __device__ __forceinline__ int freq_of_pos(int pos, int logm) {
    int k = 0, mult = 1, lg = logm, rem = pos;
    if (lg & 1) {
        --lg;
        k += (rem >> lg) * mult;
        rem &= (1 << lg) - 1;
        mult <<= 1;
    }
    while (lg > 0) {
        lg -= 2;
        k += (rem >> lg) * mult;
        rem &= (1 << lg) - 1;
        mult <<= 2;
    }
    return k;
}

// The same map with a bit reversal: reversing the bits of a 2L-bit number
// and then swapping the two bits of every pair reverses its base-4 digits.
__device__ __forceinline__ uint32_t freq_of_pos_fast(uint32_t pos, int logm) {
    uint32_t hi = 0, rest = pos;
    int lg = logm;
    if (lg & 1) {
        --lg;
        hi = rest >> lg;
        rest &= (1u << lg) - 1;
    }
    if (lg == 0) return hi;
    uint32_t r = __brev(rest) >> (32 - lg);
    r = ((r & 0x55555555u) << 1) | ((r >> 1) & 0x55555555u);
    return (logm & 1) ? hi + 2 * r : r;
}

// In-place transforms of `cnt` arrays of length M = 2^logm in shared memory
// by the whole CTA: element e of array t is base[t * ts + e * es].  With
// `fast_t`, consecutive threads take consecutive arrays (for arrays stored
// side by side, es = cnt); otherwise consecutive elements of one array.
// tw[e] = w_M^e (forward) or w_M^-e (inverse) for e in [0, M), with its Shoup
// quotient.
template <bool FWD, int CNT_FAST = 0>
__device__ void smem_ntt(uint32_t* base, int es, int ts, int cnt, bool fast_t, int logm,
                         const uint2* __restrict__ tw, uint32_t p) {
    if (CNT_FAST) {  // arrays side by side, CNT_FAST of them (a power of two)
        cnt = CNT_FAST;
        fast_t = true;
    }
    const int M = 1 << logm;
    const uint2 w4 = __ldg(tw + (M >> 2));  // primitive 4th root (or its inverse)
    const int quarter = M >> 2;
    const int nbf4 = cnt * quarter;
    if (FWD && (logm & 1)) {  // radix-2 stage, span M/2
        const int h = M >> 1;
        for (int idx = threadIdx.x; idx < cnt * h; idx += blockDim.x) {
            const int t = CNT_FAST ? (idx & (CNT_FAST - 1)) : fast_t ? idx % cnt : idx >> (logm - 1);
            const int j = CNT_FAST ? (idx / CNT_FAST) : fast_t ? idx / cnt : idx & (h - 1);
            uint32_t* x = base + t * ts;
            const uint32_t u = x[j * es], v = x[(j + h) * es];
            x[j * es] = add_p(u, v, p);
            x[(j + h) * es] = mul_shoup(sub_p(u, v, p), __ldg(tw + j), p);
        }
        __syncthreads();
    }
    const int smax = (logm & 1) ? (M >> 3) : (M >> 2);
    for (int it = 0, s = FWD ? smax : 1; FWD ? s >= 1 : s <= smax; ++it, s = FWD ? (s >> 2) : (s << 2)) {
        const int lgs = FWD ? (logm & 1 ? logm - 3 : logm - 2) - 2 * it : 2 * it;  // log2 s
        const int lgstep = logm - 2 - lgs;  // twiddle exponent step M/(4s)
        for (int idx = threadIdx.x; idx < nbf4; idx += blockDim.x) {
            const int t = CNT_FAST ? (idx & (CNT_FAST - 1)) : fast_t ? idx % cnt : idx >> (logm - 2);
            const int b = CNT_FAST ? (idx / CNT_FAST) : fast_t ? idx / cnt : idx & (quarter - 1);
            const int blk = b >> lgs, j = b & (s - 1);
            uint32_t* x = base + t * ts + ((blk << (lgs + 2)) + j) * es;
            const int e = j << lgstep;
            const int se = s * es;
            uint32_t x0 = x[0], x1 = x[se], x2 = x[2 * se], x3 = x[3 * se];
            if (!FWD) {  // decimation in time: twiddle the inputs
                x1 = mul_shoup(x1, __ldg(tw + e), p);
                x2 = mul_shoup(x2, __ldg(tw + 2 * e), p);
                x3 = mul_shoup(x3, __ldg(tw + 3 * e), p);
            }
            const uint32_t t0 = add_p(x0, x2, p), t1 = sub_p(x0, x2, p);
            const uint32_t t2 = add_p(x1, x3, p), t3 = mul_shoup(sub_p(x1, x3, p), w4, p);
            uint32_t z0 = add_p(t0, t2, p), z2 = sub_p(t0, t2, p);
            uint32_t z1 = add_p(t1, t3, p), z3 = sub_p(t1, t3, p);
            if (FWD) {  // decimation in frequency: twiddle the outputs
                z1 = mul_shoup(z1, __ldg(tw + e), p);
                z2 = mul_shoup(z2, __ldg(tw + 2 * e), p);
                z3 = mul_shoup(z3, __ldg(tw + 3 * e), p);
            }
            x[0] = z0; x[se] = z1; x[2 * se] = z2; x[3 * se] = z3;
        }
        __syncthreads();
    }
    if (!FWD && (logm & 1)) {  // radix-2 stage, span M/2
        const int h = M >> 1;
        for (int idx = threadIdx.x; idx < cnt * h; idx += blockDim.x) {
            const int t = CNT_FAST ? (idx & (CNT_FAST - 1)) : fast_t ? idx % cnt : idx >> (logm - 1);
            const int j = CNT_FAST ? (idx / CNT_FAST) : fast_t ? idx / cnt : idx & (h - 1);
            uint32_t* x = base + t * ts;
            const uint32_t u = x[j * es], v = mul_shoup(x[(j + h) * es], __ldg(tw + j), p);
            x[j * es] = add_p(u, v, p);
            x[(j + h) * es] = sub_p(u, v, p);
        }
        __syncthreads();
    }
}

// A radix-4 butterfly with the twiddles given (tw1..tw3 = w^e, w^2e, w^3e; none when
// !on), lazy: inputs and outputs in [0, 2p).  Forward (decimation in frequency):
// t0 = x0 + x2, t1 = x0 - x2, t2 = x1 + x3, t3 = (x1 - x3) w4, then z0 = t0 + t2,
// z1 = (t1 + t3) w^e, z2 = (t0 - t2) w^2e, z3 = (t1 - t3) w^3e; inverse (in time): the
// inputs x1..x3 twiddled first, the same network without output twiddles.
template <bool FWD>
__device__ __forceinline__ void bf4t(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3, uint2 w4, uint2 tw1,
                                     uint2 tw2, uint2 tw3, bool on, uint32_t p) {
    const uint32_t p2 = 2 * p;
    if (!FWD && on) {
        x1 = mul_shoup_lz(x1, tw1, p);
        x2 = mul_shoup_lz(x2, tw2, p);
        x3 = mul_shoup_lz(x3, tw3, p);
    }
    const uint32_t t0 = r2p(x0 + x2, p2), t1 = r2p(x0 - x2 + p2, p2);
    const uint32_t t2 = r2p(x1 + x3, p2), t3 = mul_shoup_lz(x1 - x3 + p2, w4, p);
    x0 = r2p(t0 + t2, p2);
    if (FWD && on) {
        x1 = mul_shoup_lz(t1 + t3, tw1, p);
        x2 = mul_shoup_lz(t0 - t2 + p2, tw2, p);
        x3 = mul_shoup_lz(t1 - t3 + p2, tw3, p);
    } else {
        x1 = r2p(t1 + t3, p2);
        x2 = r2p(t0 - t2 + p2, p2);
        x3 = r2p(t1 - t3 + p2, p2);
    }
}

// One radix-4 butterfly on registers with twiddle exponent e (the same
// network as smem_ntt's), lazy.  The exponent varies across the lanes of a
// warp here, so e = 0 is not special-cased: it multiplies by the table's
// entry 0 (= 1, whose Shoup product also lands in [0, 2p)) and no lane
// takes another path.
template <bool FWD>
__device__ __forceinline__ void bf4(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3, uint2 w4,
                                    const uint2* __restrict__ tw, int e, uint32_t p) {
    bf4t<FWD>(x0, x1, x2, x3, w4, __ldg(tw + e), __ldg(tw + 2 * e), __ldg(tw + 3 * e), true, p);
}

// One radix-2 butterfly with twiddle exponent e (smem_ntt's radix-2 stage).
// (lazy: inputs and outputs in [0, 2p))
template <bool FWD>
__device__ __forceinline__ void bf2(uint32_t& u, uint32_t& v, const uint2* __restrict__ tw, int e, uint32_t p) {
    const uint32_t p2 = 2 * p;
    const uint2 tv = __ldg(tw + e);  // (e = 0: entry 0 = 1, as in bf4)
    if (FWD) {
        const uint32_t d = u - v + p2;  // (0, 4p)
        u = r2p(u + v, p2);
        v = mul_shoup_lz(d, tv, p);
    } else {
        const uint32_t w = mul_shoup_lz(v, tv, p);
        v = r2p(u - w + p2, p2);
        u = r2p(u + w, p2);
    }
}

// Column transforms in shared memory by register stages: the levels of
// smem_ntt (the same butterflies and twiddles, so the same output order),
// two at a time.  A stage pairs a level of span s_large and radix RL with the
// next level of span s_small = s_large / RS and radix RS; a thread takes the
// RS * RL elements base + j + ks s_small + kl s_large (j < s_small) of one
// column into registers, applies both levels (forward: large span first,
// inverse: small span first) and writes them back, so each pair of levels
// costs one read and one write of shared memory.  Columns are side by side,
// with one pad row after every 16 rows: element n1 of column c is
// sh[cphys(n1) * COLS + c], cphys(n1) = n1 + n1 / 16, so that the stage whose
// small span is 1 (16 consecutive rows per unit) reads the units of a warp
// from distinct banks.  The column length 2^LOGM and every span are
// compile-time constants, and so is each element's offset from its unit's
// first element: for every unit of every stage, base mod 16 plus the offset
// K mod 16 stays below 16 (all spans are powers of 4, and a unit's elements
// below span 16 share one group of 16 rows), so cphys(base + K) =
// cphys(base) + K + K / 16.
__device__ __forceinline__ int cphys(int n1) { return n1 + (n1 >> 4); }
template <bool FWD, int RS, int RL, int COLS, int LOGM, int LG_SS>
__device__ __forceinline__ void col_stage(uint32_t* sh, const uint2* __restrict__ tw, uint2 w4, uint32_t p) {
    constexpr int R = RS * RL;
    constexpr int SS = 1 << LG_SS;
    constexpr int LG_SL = LG_SS + (RS == 4 ? 2 : 0);
    constexpr int LG_BLK = LG_SL + (RL == 4 ? 2 : 1);
    constexpr int NUNITS = COLS << (LOGM - (RS == 4 ? 2 : 0) - (RL == 4 ? 2 : 1));
#pragma unroll 1
    for (int u = threadIdx.x; u < NUNITS; u += NTT_THREADS) {
        const int c = u & (COLS - 1), v = u / COLS;
        const int j = v & (SS - 1), blk = v >> LG_SS;
        const int base = (blk << LG_BLK) + j;
        if (!PM_CHK(base + ((RS - 1) << LG_SS) + ((RL - 1) << LG_SL) < (1 << LOGM))) continue;
        uint32_t* pb = sh + cphys(base) * COLS + c;
        uint32_t r[R];
#pragma unroll
        for (int kl = 0; kl < RL; ++kl)
#pragma unroll
            for (int ks = 0; ks < RS; ++ks) {
                const int K = (ks << LG_SS) + (kl << LG_SL);
                r[ks + RS * kl] = pb[(K + (K >> 4)) * COLS];
            }
        // the level of span s_large: offsets j + ks s_small in its blocks
        auto large = [&]() {
#pragma unroll
            for (int ks = 0; ks < RS; ++ks) {
                const int jl = j + (ks << LG_SS);
                if constexpr (RL == 4 && RS == 1 && LG_SL == 0) {  // a single level of span 1: no twiddles
                    bf4t<FWD>(r[ks], r[ks + RS], r[ks + 2 * RS], r[ks + 3 * RS], w4, w4, w4, w4, false, p);
                } else if constexpr (RL == 4) {
                    const int e = jl << (LOGM - 2 - LG_SL);
                    bf4<FWD>(r[ks], r[ks + RS], r[ks + 2 * RS], r[ks + 3 * RS], w4, tw, e, p);
                } else {
                    bf2<FWD>(r[ks], r[ks + RS], tw, jl, p);  // span M/2: twiddle exponent = offset
                }
            }
        };
        // the level of span s_small (radix 4): offset j in its blocks (span 1: j = 0, every twiddle
        // is w^0 = 1 and the butterflies take none)
        auto small = [&]() {
            if constexpr (RS == 4 && LG_SS == 0) {
#pragma unroll
                for (int kl = 0; kl < RL; ++kl)
                    bf4t<FWD>(r[RS * kl], r[RS * kl + 1], r[RS * kl + 2], r[RS * kl + 3], w4, w4, w4, w4, false, p);
            } else if constexpr (RS == 4) {
                const int e = j << (LOGM - 2 - LG_SS);
#pragma unroll
                for (int kl = 0; kl < RL; ++kl) bf4<FWD>(r[RS * kl], r[RS * kl + 1], r[RS * kl + 2], r[RS * kl + 3], w4, tw, e, p);
            }
        };
        if (FWD) { large(); small(); } else { small(); large(); }
#pragma unroll
        for (int kl = 0; kl < RL; ++kl)
#pragma unroll
            for (int ks = 0; ks < RS; ++ks) {
                const int K = (ks << LG_SS) + (kl << LG_SL);
                pb[(K + (K >> 4)) * COLS] = r[ks + RS * kl];
            }
    }
    __syncthreads();
}

// Levels of a length-2^LOGM column transform in the forward order: radix 2 at
// span M/2 first when LOGM is odd, then radix 4 from span M/4 (or M/8) down to 1.
__host__ __device__ constexpr int col_nlev(int logm) { return (logm & 1) + (logm >> 1); }
__host__ __device__ constexpr int col_lv_lg(int logm, int i) {  // log2 of level i's span
    return (logm & 1) ? (i == 0 ? logm - 1 : logm - 1 - 2 * i) : logm - 2 - 2 * i;
}
__host__ __device__ constexpr bool col_lv_r2(int logm, int i) { return (logm & 1) && i == 0; }

// Stages ST, ST + 2, ... of the transform: the forward order takes levels ST and
// ST + 1, the inverse the mirror ones.
template <bool FWD, int COLS, int LOGM, int ST>
__device__ __forceinline__ void col_stages(uint32_t* sh, const uint2* __restrict__ tw, uint2 w4, uint32_t p) {
    constexpr int NLEV = col_nlev(LOGM);
    if constexpr (ST < NLEV) {
        constexpr int A = FWD ? ST : NLEV - 1 - ST;   // first level executed
        if constexpr (ST + 1 < NLEV) {
            constexpr int B = FWD ? ST + 1 : NLEV - 2 - ST;
            constexpr int LARGE = FWD ? A : B, SMALL = FWD ? B : A;
            col_stage<FWD, 4, col_lv_r2(LOGM, LARGE) ? 2 : 4, COLS, LOGM, col_lv_lg(LOGM, SMALL)>(sh, tw, w4, p);
        } else {
            col_stage<FWD, 1, col_lv_r2(LOGM, A) ? 2 : 4, COLS, LOGM, col_lv_lg(LOGM, A)>(sh, tw, w4, p);
        }
        col_stages<FWD, COLS, LOGM, ST + 2>(sh, tw, w4, p);
    }
}

// The transforms of COLS side-by-side columns of length 2^LOGM (1 <= LOGM).
template <bool FWD, int COLS, int LOGM>
__device__ __forceinline__ void col_transform(uint32_t* sh, const uint2* __restrict__ tw, uint32_t p) {
    const uint2 w4 = LOGM >= 2 ? __ldg(tw + (1 << (LOGM >= 2 ? LOGM - 2 : 0))) : make_uint2(0, 0);
    col_stages<FWD, COLS, LOGM, 0>(sh, tw, w4, p);
}

// A length-4096 transform as three radix-16 stages, each two radix-4 levels
// done in registers by 256 threads holding 16 elements (the levels of
// smem_ntt with logm = 12, grouped by the elements they touch):
//   stage 1: elements t + 256 l      (levels s = 1024, 256)
//   stage 2: elements B + t' + 16 l   (B = 256 (t / 16), t' = t mod 16; levels s = 64, 16)
//   stage 3: elements 16 t + l        (levels s = 4, 1)
// Forward runs stages 1, 2, 3 (levels large to small); the inverse 3, 2, 1
// with the levels reversed.  Shared arrays use one pad word per 16 words.
__device__ __forceinline__ int rphys(int i) { return i + (i >> 4); }
constexpr int ROW_WORDS = NTT_N2 + NTT_N2 / 16;

// Twiddles of the row transforms (w = w_N2 forward, w_N2^-1 inverse), stored in the
// order the threads read them, so that a warp's load of one twiddle is one or two
// contiguous 128-byte lines (read by exponent, the second level of stage 1 and both
// levels of stage 2 would touch 8 to 24 lines per load):
//   A1[k][e]      = w^(k e),                e < 1024    stage 1, first level (e = t + 256 l0)
//   B1[k][t]      = w^(4 k t),              t < 256     stage 1, second level
//   A2[k][l0][tp] = w^(k (16 tp + 256 l0)), l0 < 4, tp < 16   stage 2, first level
//   B2[k][tp]     = w^(64 k tp),            tp < 16     stage 2, second level
// for k = 1, 2, 3 (stored at k - 1).
constexpr int RT_A1 = 0, RT_B1 = RT_A1 + 3 * 1024, RT_A2 = RT_B1 + 3 * 256, RT_B2 = RT_A2 + 3 * 64;
constexpr int RT_WORDS = RT_B2 + 3 * 16;
static_assert(RT_WORDS <= NTT_N2, "row twiddles fit the table slot");

// row_stage on NR arrays at once (the forward transforms of a's and b's rows): every
// twiddle is loaded once for all of them; stage 3's come from the kernel parameters.
template <bool FWD, int NR>
__device__ __forceinline__ void row_stage_n(int stage, uint32_t (*rs[NR])[16], uint2 w4, const uint2* __restrict__ tw,
                                            const uint2 (&c3)[3][3], uint32_t p) {
    const int t = threadIdx.x, tp = t & 15;
    auto lvA = [&]() {
#pragma unroll
        for (int l0 = 0; l0 < 4; ++l0) {
            uint2 a1, a2, a3;
            bool on = true;
            if (stage == 3) {
                on = l0 != 0;
                a1 = c3[l0 ? l0 - 1 : 0][0]; a2 = c3[l0 ? l0 - 1 : 0][1]; a3 = c3[l0 ? l0 - 1 : 0][2];
            } else {  // (exponent 0 on some lanes: multiplied by w^0 = 1, so no lane diverges)
                const uint2* q = stage == 1 ? tw + RT_A1 + t + 256 * l0 : tw + RT_A2 + 16 * l0 + tp;
                const int ks = stage == 1 ? 1024 : 64;  // stride between k = 1, 2, 3
                a1 = __ldg(q); a2 = __ldg(q + ks); a3 = __ldg(q + 2 * ks);
            }
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                uint32_t (&r)[16] = *rs[k];
                bf4t<FWD>(r[l0], r[l0 + 4], r[l0 + 8], r[l0 + 12], w4, a1, a2, a3, on, p);
            }
        }
    };
    auto lvB = [&]() {
        // stages 1 and 2: per-lane exponents (w^0 = 1 where it is 0); stage 3: none for any lane
        const bool on = stage != 3;
        uint2 a1 = make_uint2(0, 0), a2 = a1, a3 = a1;
        if (on) {
            const uint2* q = stage == 1 ? tw + RT_B1 + t : tw + RT_B2 + tp;
            const int ks = stage == 1 ? 256 : 16;
            a1 = __ldg(q); a2 = __ldg(q + ks); a3 = __ldg(q + 2 * ks);
        }
#pragma unroll
        for (int l1 = 0; l1 < 4; ++l1)
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                uint32_t (&r)[16] = *rs[k];
                bf4t<FWD>(r[4 * l1], r[4 * l1 + 1], r[4 * l1 + 2], r[4 * l1 + 3], w4, a1, a2, a3, on, p);
            }
    };
    if (FWD) { lvA(); lvB(); } else { lvB(); lvA(); }
}

// element index of register l of thread t in stage `stage`
__device__ __forceinline__ int row_index(int stage, int t, int l) {
    return stage == 1 ? t + 256 * l : stage == 2 ? 256 * (t >> 4) + (t & 15) + 16 * l : 16 * t + l;
}

// Device tables of one (p, g, log N), each entry (w, floor(w 2^32 / p)).
struct NttTables {
    const uint2 *lo, *ilo;    // w_N^e, w_N^-e, e < 4096
    const uint2 *row, *irow;  // twiddles of the row transforms (w_N2, w_N2^-1) in thread order: see RT_A1
    const uint2 *hi, *ihi;    // w_N^(4096 f), w_N^(-4096 f), f < N1 (= w_N1^f)
    const uint2 *tj;          // w_N^(j k1) at k1 * cols + j, k1 < N1, j < cols (the column block width)
    uint2 scale;              // N^-1 2^32 mod p
    uint2 rw4, riw4;          // w_N2^(N2/4), w_N2^-(N2/4)
    // the twiddles of the row transforms' third stage, the same for every thread:
    // st3[l0 - 1][k - 1] = w_N2^(256 l0 k) (ist3: w_N2^-(256 l0 k)), l0, k = 1..3
    uint2 st3[3][3], ist3[3][3];
};

// x * w_N^e (or w_N^-e) with e < N: w_N^e = lo[e mod 4096] * hi[e / 4096].  (The lazy
// form: x < 2^32, result in [0, 2p).)
__device__ __forceinline__ uint32_t mul_root_lz(uint32_t x, uint32_t e, const uint2* lo, const uint2* hi,
                                                uint32_t p) {
    return mul_shoup_lz(mul_shoup_lz(x, __ldg(lo + (e & (NTT_N2 - 1))), p), __ldg(hi + (e >> NTT_N2_LOG)), p);
}
// (w_N^e, floor(w_N^e 2^32 / p)) for e < N from the same two tables (canonical product, then its
// Shoup quotient)
__device__ __forceinline__ uint2 root_pair(uint32_t e, const uint2* lo, const uint2* hi, uint32_t p) {
    const uint32_t w = mul_shoup(__ldg(lo + (e & (NTT_N2 - 1))).x, __ldg(hi + (e >> NTT_N2_LOG)), p);
    return make_uint2(w, (uint32_t)(((uint64_t)w << 32) / p));
}

// ---- N < 1024, or N <= 4096 with a prime of 2-adic order below 12: one CTA, length-N transforms in
// shared memory ----
__global__ void __launch_bounds__(NTT_THREADS) ntt_small_kernel(
    const uint32_t* __restrict__ a, int n, const uint32_t* __restrict__ b, int m,
    uint32_t* __restrict__ c, int logn, NttTables tb, NttMod md) {
    extern __shared__ uint32_t sh[];
    const int N = 1 << logn, L = n + m - 1;
    uint32_t* sa = sh;
    uint32_t* sb = sh + N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        sa[i] = i < n ? a[i] : 0u;
        sb[i] = i < m ? b[i] : 0u;
    }
    __syncthreads();
    smem_ntt<true>(sh, 1, N, 2, false, logn, tb.lo, md.p);
    for (int i = threadIdx.x; i < N; i += blockDim.x) sa[i] = mul_mont(sa[i], sb[i], md);
    __syncthreads();
    smem_ntt<false>(sa, 1, N, 1, false, logn, tb.ilo, md.p);
    for (int i = threadIdx.x; i < L; i += blockDim.x) c[i] = mul_shoup(sa[i], tb.scale, md.p);
}

__device__ __forceinline__ void cp_async4_ntt(uint32_t* dst, const uint32_t* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

// ---- four-step pass 1: forward column transforms of a (y = 0) and b (y = 1) ----
// A CTA takes COLS adjacent columns of length N1 = 2^LOG1; shared memory holds
// them row by row ([n1][COLS]), so loads and stores touch 4 COLS contiguous
// bytes per row and the butterflies of the COLS columns run side by side.
template <int COLS, int LOG1>
__global__ void __launch_bounds__(NTT_THREADS, NTT_COL_MINB) ntt_col_fwd_kernel(
    const uint32_t* __restrict__ a, int n, const uint32_t* __restrict__ b, int m,
    uint32_t* __restrict__ ta, uint32_t* __restrict__ tb_out, NttTables tb, NttMod md) {
    constexpr int N1 = 1 << LOG1;
    extern __shared__ uint32_t sh[];
    pdl_trigger();  // the row pass may be placed now; it waits for this pass to end
    if (!PM_CHK((blockIdx.x + 1) * COLS <= NTT_N2 && blockIdx.y < 2)) return;  // (uniform: before any barrier)
    const uint32_t* x = blockIdx.y == 0 ? a : b;
    const int len = blockIdx.y == 0 ? n : m;
    uint32_t* out = blockIdx.y == 0 ? ta : tb_out;
    const int c0 = blockIdx.x * COLS;
#pragma unroll 4
    for (int idx = threadIdx.x; idx < COLS * N1; idx += NTT_THREADS) {
        const int j = idx % COLS, n1 = idx / COLS;
        const int g = n1 * NTT_N2 + c0 + j;
        cp_async4_ntt(sh + cphys(n1) * COLS + j, x + (g < len ? g : 0), g < len);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    col_transform<true, COLS, LOG1>(sh, tb.hi, md.p);
    // the twist w_N^((c0 + j) k1) = w_N^(c0 k1) (two table factors, one pair per position: 4 per
    // warp) times w_N^(j k1) (tb.tj, j fastest: 4 runs of COLS entries per warp), so that a warp's
    // loads touch 4 lines each; (c0 + j) k1 < 4096 N1 = N, so no exponent wraps
#pragma unroll 4
    for (int idx = threadIdx.x; idx < COLS * N1; idx += NTT_THREADS) {
        const int j = idx % COLS, pos = idx / COLS;
        const uint32_t k1 = freq_of_pos_fast((uint32_t)pos, LOG1);
        const uint32_t e0 = (uint32_t)c0 * k1;
        const uint32_t x = mul_shoup_lz(sh[cphys(pos) * COLS + j], __ldg(tb.lo + (e0 & (NTT_N2 - 1))), md.p);
        out[(size_t)pos * NTT_N2 + c0 + j] =
            mul_shoup_lz(mul_shoup_lz(x, __ldg(tb.hi + (e0 >> NTT_N2_LOG)), md.p), __ldg(tb.tj + k1 * COLS + j), md.p);
    }
}

// The product of one row pair in registers (the pass-2 work of a row): on entry thread t holds
// elements t + 256 l (l < 16) of the two length-4096 rows in r and q, on exit the inverse
// transform of their transforms' pointwise product (Montgomery: times 2^-32) in r, in the same
// positions; sA and sB are the CTA's exchange arrays.
__device__ __forceinline__ void row_product(uint32_t (&r)[16], uint32_t (&q)[16], uint32_t* sA, uint32_t* sB,
                                            const NttTables& tb, const NttMod& md) {
    const int t = threadIdx.x;
    const uint32_t p = md.p;
    const uint2 w4 = tb.rw4, iw4 = tb.riw4;
    uint32_t (*rq[2])[16] = {&r, &q};
    uint32_t (*ro[1])[16] = {&r};
    row_stage_n<true, 2>(1, rq, w4, tb.row, tb.st3, p);
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        sA[rphys(t + 256 * l)] = r[l];
        sB[rphys(t + 256 * l)] = q[l];
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        r[l] = sA[rphys(row_index(2, t, l))];
        q[l] = sB[rphys(row_index(2, t, l))];
    }
    row_stage_n<true, 2>(2, rq, w4, tb.row, tb.st3, p);
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        sA[rphys(row_index(2, t, l))] = r[l];
        sB[rphys(row_index(2, t, l))] = q[l];
    }
    __syncthreads();
    // stage 3, the pointwise product and the first inverse stage stay in registers
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        r[l] = sA[rphys(16 * t + l)];
        q[l] = sB[rphys(16 * t + l)];
    }
    row_stage_n<true, 2>(3, rq, w4, tb.row, tb.st3, p);
#pragma unroll
    for (int l = 0; l < 16; ++l) r[l] = mul_mont_lz(r[l], q[l], md);
    row_stage_n<false, 1>(3, ro, iw4, tb.irow, tb.ist3, p);
    __syncthreads();  // every thread has read its stage-3 inputs from sA
#pragma unroll
    for (int l = 0; l < 16; ++l) sA[rphys(16 * t + l)] = r[l];
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) r[l] = sA[rphys(row_index(2, t, l))];
    row_stage_n<false, 1>(2, ro, iw4, tb.irow, tb.ist3, p);
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) sA[rphys(row_index(2, t, l))] = r[l];
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) r[l] = sA[rphys(t + 256 * l)];
    row_stage_n<false, 1>(1, ro, iw4, tb.irow, tb.ist3, p);
}

// ---- four-step pass 2: per row, forward row transforms, product, inverse ----
__global__ void __launch_bounds__(256, NTT_ROW_MINB) ntt_row_kernel(uint32_t* __restrict__ ta,
                                                      const uint32_t* __restrict__ tbuf,
                                                      int logn1, NttTables tb, NttMod md) {
    __shared__ uint32_t sA[ROW_WORDS];
    __shared__ uint32_t sB[ROW_WORDS];
    const int t = threadIdx.x;
    const size_t r0 = (size_t)blockIdx.x * NTT_N2;
    pdl_wait();  // the column pass's transforms
    pdl_trigger();
    if (!PM_CHK(blockIdx.x < (1u << logn1) && blockDim.x == 256)) return;  // (uniform: before any barrier)
    const uint32_t p = md.p;
    const uint32_t k1 = freq_of_pos_fast(blockIdx.x, logn1);
    const uint64_t nmask = ((((uint64_t)1) << logn1) << NTT_N2_LOG) - 1;
    // the final twist by w_N^-(i k1), i = t + 256 l, as w_N^-(256 l k1) (one per l, for the whole
    // CTA: sC, read after the barriers below) times w_N^-(t k1) (one per thread)
    __shared__ uint2 sC[16];
    if (t < 16) sC[t] = root_pair((uint32_t)((256ull * t * k1) & nmask), tb.ilo, tb.ihi, p);
    uint32_t r[16], q[16];
    // stage 1 of both rows, straight from global memory
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        r[l] = ta[r0 + t + 256 * l];
        q[l] = tbuf[r0 + t + 256 * l];
    }
    row_product(r, q, sA, sB, tb, md);
    const uint2 bt = root_pair((uint32_t)(((uint64_t)t * k1) & nmask), tb.ilo, tb.ihi, p);
#pragma unroll
    for (int l = 0; l < 16; ++l) ta[r0 + t + 256 * l] = mul_shoup_lz(mul_shoup_lz(r[l], sC[l], p), bt, p);
}

// ---- products with N <= 4096: one row pair in one CTA ----
// The length-4096 transform of the row pass, on a and b zero-padded to 4096 words (a cyclic product
// of length 4096 is the whole product when n + m - 1 <= 4096), then the scale N^-1 2^32 and the
// store of the n + m - 1 output words.
__global__ void __launch_bounds__(256) ntt_one_row_kernel(const uint32_t* __restrict__ a, int n,
                                                          const uint32_t* __restrict__ b, int m,
                                                          uint32_t* __restrict__ c, int L, NttTables tb, NttMod md) {
    __shared__ uint32_t sA[ROW_WORDS];
    __shared__ uint32_t sB[ROW_WORDS];
    const int t = threadIdx.x;
    if (!PM_CHK(blockDim.x == 256 && n + m - 1 <= NTT_N2)) return;  // (uniform: before any barrier)
    uint32_t r[16], q[16];
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        const int i = t + 256 * l;
        r[l] = i < n ? a[i] : 0u;
        q[l] = i < m ? b[i] : 0u;
    }
    row_product(r, q, sA, sB, tb, md);
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        const int i = t + 256 * l;
        if (i < L) c[i] = mul_shoup(r[l], tb.scale, md.p);
    }
}

// ---- four-step pass 3: inverse column transforms, scale, store ----
template <int COLS, int LOG1>
__global__ void __launch_bounds__(NTT_THREADS, NTT_COL_MINB) ntt_col_inv_kernel(const uint32_t* __restrict__ ta,
                                                                  uint32_t* __restrict__ c, int L,
                                                                  NttTables tb, NttMod md) {
    constexpr int N1 = 1 << LOG1;
    extern __shared__ uint32_t sh[];
    const int c0 = blockIdx.x * COLS;
    pdl_wait();  // the row pass's products
    if (!PM_CHK((blockIdx.x + 1) * COLS <= NTT_N2)) return;  // (uniform: before any barrier)
#pragma unroll 4
    for (int idx = threadIdx.x; idx < COLS * N1; idx += NTT_THREADS) {
        const int j = idx % COLS, pos = idx / COLS;
        cp_async4_ntt(sh + cphys(pos) * COLS + j, ta + (size_t)pos * NTT_N2 + c0 + j, true);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    col_transform<false, COLS, LOG1>(sh, tb.ihi, md.p);
#pragma unroll 4
    for (int idx = threadIdx.x; idx < COLS * N1; idx += NTT_THREADS) {
        const int j = idx % COLS, n1 = idx / COLS;
        const int64_t g = (int64_t)n1 * NTT_N2 + c0 + j;
        if (g < L) c[g] = mul_shoup(sh[cphys(n1) * COLS + j], tb.scale, md.p);
    }
}

// The column kernels of every log2 N1 = 1 .. 12 (blocks of 8 columns from
// NTT_COLS8_LOG on, else 16).
template <int LOG1>
constexpr int col_block() { return LOG1 >= NTT_COLS8_LOG ? 8 : 16; }
using ColFwdFn = void (*)(const uint32_t*, int, const uint32_t*, int, uint32_t*, uint32_t*, NttTables, NttMod);
using ColInvFn = void (*)(const uint32_t*, uint32_t*, int, NttTables, NttMod);
template <int... L>
struct ColKernels {
    static constexpr ColFwdFn fwd[sizeof...(L)] = {ntt_col_fwd_kernel<col_block<L>(), L>...};
    static constexpr ColInvFn inv[sizeof...(L)] = {ntt_col_inv_kernel<col_block<L>(), L>...};
    static constexpr int cols[sizeof...(L)] = {col_block<L>()...};
};
using ColTable = ColKernels<1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12>;
static_assert(NTT_MAX_LOG - NTT_N2_LOG == 12, "column kernels for log2 N1 = 1 .. 12");

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static uint32_t powmod_h(uint64_t b, uint64_t e, uint32_t p) {
    uint64_t r = 1 % p;
    b %= p;
    while (e) {
        if (e & 1) r = r * b % p;
        b = b * b % p;
        e >>= 1;
    }
    return (uint32_t)r;
}

static uint2 shoup_pair(uint32_t w, uint32_t p) {
    return make_uint2(w, (uint32_t)((((uint64_t)w) << 32) / p));
}

struct TableSet {
    uint2* dev = nullptr;
    NttTables t{};
};

static std::mutex g_tab_mutex;
static std::map<std::tuple<int, uint32_t, uint32_t, int>, TableSet> g_tables;

// Builds (once) the twiddle tables of (device, p, g, logn) with a synchronous copy.
static pm_status get_tables(int dev, uint32_t p, uint32_t g, int logn, cudaStream_t st, NttTables* out) {
    std::lock_guard<std::mutex> lock(g_tab_mutex);
    auto key = std::make_tuple(dev, p, g, logn);
    auto it = g_tables.find(key);
    if (it != g_tables.end()) {
        *out = it->second.t;
        return PM_OK;
    }
    if (is_capturing(st)) return PM_ERR_UNSUPPORTED;
    const uint64_t N = 1ull << logn;
    const uint32_t w = powmod_h(g, (uint64_t)(p - 1) / N, p);
    if (N >= 2 && powmod_h(w, N / 2, p) != p - 1) return PM_ERR_UNSUPPORTED;  // not of order N
    const uint32_t wi = powmod_h(w, p - 2, p);
    const int n1 = logn > NTT_N2_LOG ? (int)(N >> NTT_N2_LOG) : 1;
    const int tcols = logn > NTT_N2_LOG ? ColTable::cols[logn - NTT_N2_LOG - 1] : 0;  // columns per block
    const size_t words = 4 * NTT_N2 + 2 * (size_t)n1 + (size_t)tcols * n1;
    std::vector<uint2> h(words);
    uint2* lo = h.data();
    uint2* ilo = lo + NTT_N2;
    uint2* row = ilo + NTT_N2;
    uint2* irow = row + NTT_N2;
    uint2* hi = irow + NTT_N2;
    uint2* ihi = hi + n1;
    uint2* tj = ihi + n1;
    for (int k1 = 0; k1 < (tcols ? n1 : 0); ++k1)
        for (int j = 0; j < tcols; ++j) tj[(size_t)k1 * tcols + j] = shoup_pair(powmod_h(w, ((uint64_t)j * k1) % N, p), p);
    for (int e = 0; e < NTT_N2; ++e) {
        lo[e] = shoup_pair(powmod_h(w, (uint64_t)e % N, p), p);
        ilo[e] = shoup_pair(powmod_h(wi, (uint64_t)e % N, p), p);
    }
    if (logn >= NTT_N2_LOG) {  // the row transforms' twiddles in thread order (RT_A1 ...)
        const uint32_t w2 = powmod_h(w, (uint64_t)n1, p), w2i = powmod_h(wi, (uint64_t)n1, p);  // w_N2, w_N2^-1
        auto fill = [&](uint2* T, uint32_t base) {
            auto pw = [&](uint64_t x) { return shoup_pair(powmod_h(base, x % NTT_N2, p), p); };
            for (int k = 1; k <= 3; ++k) {
                for (int e = 0; e < 1024; ++e) T[RT_A1 + (k - 1) * 1024 + e] = pw((uint64_t)k * e);
                for (int t = 0; t < 256; ++t) T[RT_B1 + (k - 1) * 256 + t] = pw(4ull * k * t);
                for (int l0 = 0; l0 < 4; ++l0)
                    for (int tp = 0; tp < 16; ++tp)
                        T[RT_A2 + ((k - 1) * 4 + l0) * 16 + tp] = pw((uint64_t)k * (16 * tp + 256 * l0));
                for (int tp = 0; tp < 16; ++tp) T[RT_B2 + (k - 1) * 16 + tp] = pw(64ull * k * tp);
            }
        };
        fill(row, w2);
        fill(irow, w2i);
    }
    for (int f = 0; f < n1; ++f) {
        hi[f] = shoup_pair(powmod_h(w, ((uint64_t)NTT_N2 * f) % N, p), p);
        ihi[f] = shoup_pair(powmod_h(wi, ((uint64_t)NTT_N2 * f) % N, p), p);
    }
    TableSet ts;
    if (dev_alloc((void**)&ts.dev, words * sizeof(uint2)) != cudaSuccess) {
        cudaGetLastError();
        return PM_ERR_NOMEM;
    }
    cudaError_t e = cudaMemcpy(ts.dev, h.data(), words * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(ts.dev);
        return cuda_fail(e);
    }
    ts.t.lo = ts.dev;
    ts.t.ilo = ts.dev + NTT_N2;
    ts.t.row = ts.dev + 2 * NTT_N2;
    ts.t.irow = ts.dev + 3 * NTT_N2;
    ts.t.hi = ts.dev + 4 * NTT_N2;
    ts.t.ihi = ts.t.hi + n1;
    ts.t.tj = ts.t.ihi + n1;
    // N^-1 * 2^32 mod p cancels the Montgomery factor of the pointwise product
    const uint32_t ninv = powmod_h(N % p, p - 2, p);
    const uint32_t r32 = (uint32_t)((1ull << 32) % p);
    ts.t.scale = shoup_pair((uint32_t)((uint64_t)ninv * r32 % p), p);
    if (logn >= NTT_N2_LOG) {
        const uint32_t w2 = powmod_h(w, (uint64_t)n1, p), w2i = powmod_h(wi, (uint64_t)n1, p);  // w_N2, w_N2^-1
        for (int l0 = 1; l0 <= 3; ++l0)
            for (int k = 1; k <= 3; ++k) {
                ts.t.st3[l0 - 1][k - 1] = shoup_pair(powmod_h(w2, (uint64_t)(256 * l0 * k), p), p);
                ts.t.ist3[l0 - 1][k - 1] = shoup_pair(powmod_h(w2i, (uint64_t)(256 * l0 * k), p), p);
            }
        ts.t.rw4 = shoup_pair(powmod_h(w2, NTT_N2 / 4, p), p);
        ts.t.riw4 = shoup_pair(powmod_h(w2i, NTT_N2 / 4, p), p);
    }
    g_tables[key] = ts;
    *out = ts.t;
    return PM_OK;
}

void release_ntt_tables() {
    std::lock_guard<std::mutex> lock(g_tab_mutex);
    for (auto& kv : g_tables) cudaFree(kv.second.dev);
    g_tables.clear();
}

pm_status launch_ntt(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* c,
                     uint32_t p, uint32_t g, cudaStream_t st, DeviceWorkspace* ws) {
    if (g == 0) {
        if (p != 469762049u) return PM_ERR_UNSUPPORTED;  // generator known for 7*2^26+1 only
        g = 3;
    }
    if (g >= p) return PM_ERR_INVALID_ARG;
    const int64_t L = n + m - 1;
    int logn = 0;
    while ((1ll << logn) < L) ++logn;
    if (logn > NTT_MAX_LOG) return PM_ERR_RANGE;
    if (logn < 2) logn = 2;
    if ((uint64_t)(p - 1) % (1ull << logn) != 0) return PM_ERR_UNSUPPORTED;
    // 1024 <= N <= 4096 takes the length-4096 row transform when p allows it (4096 | p - 1): one
    // CTA, 12.9 us on GB300 at every such N, where the length-N transform in shared memory took
    // 19 us (N = 2048) and 31 us (N = 4096); below 1024 points the latter is faster (8.9 us at
    // N = 32, 10.9 us at N = 512) and keeps them, as it keeps primes of 2-adic order below 12
    const bool one_row = logn >= 10 && logn <= NTT_N2_LOG && (p - 1) % NTT_N2 == 0;
    NttTables tb;
    pm_status rc = get_tables(ws->device, p, g, one_row ? NTT_N2_LOG : logn, st, &tb);
    if (rc != PM_OK) return rc;
    cudaError_t eb = chk_bind(ws);
    if (eb != cudaSuccess) return cuda_fail(eb);
    NttMod md;
    md.p = p;
    uint32_t inv = 1;  // p^-1 mod 2^32 by Newton iteration (p odd)
    for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
    md.pinv_neg = 0u - inv;
    cudaError_t e;
    if (one_row) {
        ntt_one_row_kernel<<<1, 256, 0, st>>>(a, (int)n, b, (int)m, c, (int)L, tb, md);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
        count_launches(1);
        return PM_OK;
    }
    if (logn <= NTT_N2_LOG) {
        const size_t smem = 2 * sizeof(uint32_t) * ((size_t)1 << logn);
        static int done[64] = {};
        if (!done[ws->device]) {
            e = cudaFuncSetAttribute(ntt_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * sizeof(uint32_t) * NTT_N2));
            if (e != cudaSuccess) return cuda_fail(e);
            done[ws->device] = 1;
        }
        ntt_small_kernel<<<1, NTT_THREADS, smem, st>>>(a, (int)n, b, (int)m, c, logn, tb, md);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
        count_launches(1);
        return PM_OK;
    }
    const int logn1 = logn - NTT_N2_LOG;
    const size_t N = (size_t)1 << logn;
    StreamScratch* sc = nullptr;
    rc = stream_scratch(ws, st, &sc);
    if (rc != PM_OK) return rc;
    rc = ensure_scratch(&sc->ntt, &sc->ntt_bytes, 2 * N * sizeof(uint32_t), st, false);
    if (rc != PM_OK) return rc;
    uint32_t* ta = reinterpret_cast<uint32_t*>(sc->ntt);
    uint32_t* tbuf = ta + N;
    const int cols = ColTable::cols[logn1 - 1];  // a CTA's columns: cols * N1 words of shared memory
    const size_t col_rows = ((size_t)1 << logn1) + ((size_t)1 << logn1) / 16;  // with a pad row per 16
    const size_t col_smem = sizeof(uint32_t) * (size_t)cols * col_rows;
    static int col_done[64] = {};
    if (!col_done[ws->device]) {
        for (int l = 1; l <= NTT_MAX_LOG - NTT_N2_LOG; ++l) {
            const int rows = (1 << l) + (1 << l) / 16;
            const int bytes = (int)(sizeof(uint32_t) * ColTable::cols[l - 1] * rows);
            e = cudaFuncSetAttribute((const void*)ColTable::fwd[l - 1], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     bytes);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute((const void*)ColTable::inv[l - 1],
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        col_done[ws->device] = 1;
    }
    ColTable::fwd[logn1 - 1]<<<dim3(NTT_N2 / cols, 2), NTT_THREADS, col_smem, st>>>(a, (int)n, b, (int)m, ta, tbuf,
                                                                                  tb, md);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_dep(ntt_row_kernel, dim3(1u << logn1), dim3(256), 0, st, ta, (const uint32_t*)tbuf, logn1, tb,
                       md);
    if (e == cudaSuccess)
        e = launch_dep(ColTable::inv[logn1 - 1], dim3(NTT_N2 / cols), dim3(NTT_THREADS), col_smem, st,
                       (const uint32_t*)ta, c, (int)L, tb, md);
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(3);
    return PM_OK;
}

}  // namespace pm
