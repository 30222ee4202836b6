// Tensor-core form of the batched product (tcgen05, bf16 limbs, fp32 accumulation).
//
// The paper has no tensor-core path; this computes the same residues as the
// long multiplication of Section 5 by turning each product into a sum of
// exact small-integer matrix products.
//
// Limbs.  Coefficients are first moved to the centred range (-p/2, p/2]
// (same residue, |v| < 2^28 for p < 2^29) and written as 4 balanced base-160
// digits in [-80, 79]: d_j for b, e_i for a (an offset K = 80 (1 + 160 +
// 160^2 + 160^3) makes v + K a standard base-160 number below 160^4); bf16
// holds them exactly.  Then
//     c = sum_{i<4, j<4} 160^i 160^j (e_i * d_j)   (mod p),
// and every entry of a digit convolution e_i * d_j accumulated over a group of
// shifts is a sum of products of magnitude <= 80 * 80 = 6400, one for each
// index of b the group's shifts reach (at most min(n, m), and at most 32 per
// shift): with at most 2592 terms it stays below 2^24 in magnitude and the
// tensor core's fp32 accumulation is exact.  A tile whose shifts reach more
// than 2592 indices of both operands (min(n, m) > 2592) is done in K-groups of
// at most 81 shifts, each accumulated on its own and reduced mod p, the later
// groups added onto the earlier groups' residues in the epilogue.  16 limb
// products per modular MAC.  (The build option PM_TC_ENC=0 keeps the earlier
// encoding: 5 base-64 digits of a in [-32, 31] x 4 base-256 digits of b, 20
// limb products, 4096 terms per group, tiles of 48 blocks.  tcgen05 kind::i8
// would hold larger limbs, but ptxas rejects it for sm_103a.)
//
// Matrix form (T = 32 outputs per block, block I covers outputs 32 I .. 32 I + 31;
// the K index runs backwards, k' = 31 - k, in both operands):
//     D[(j, r)][(I, i)] = sum_delta sum_{k'<32} d_j[32 delta - 31 + r + k'] * e_i[32 (I - delta) + 31 - k']
//                       = (e_i * d_j)[32 I + r].
// For one shift delta this is one 128 x 256 x 32 product (two MMAs of K = 16):
// N = 256 columns are 64 output blocks times the 4 limbs of a; the a operand
// is stored once per tile as rows (J, i) = limb i of block J of a, reversed,
// and the rows shift delta needs are the same rows moved by 4 per delta, so
// its descriptor just starts 4 * 16 bytes earlier for each delta.  M = 128
// rows are the 4 limbs of b times 32 offsets r, ordered (r / 8, limb j, r mod 8)
// so that one descriptor covers all limbs: with k' reversed, the 8 x 8 core
// matrix of limb j at row group r / 8 = g and K chunk c holds
// d_j[32 delta - 31 + 8 (g + c) + row + column], a Hankel block that depends
// only on q = 4 delta + g + c.  These core matrices H_j[q] are built once per
// q in shared memory, the 4 limbs interleaved (512 bytes per q), and the
// descriptor walks them with 128 bytes between row groups (the next limb or,
// after 4 limbs, the next g) and 512 bytes between K chunks (the next q).  A
// shift thus costs 4 new core matrices per limb instead of a 128 x 32 block.
// All shifts of a K-group accumulate into one TMEM tile (256 fp32 columns x
// 128 lanes); two such tiles alternate.  Every MMA spans the full width: the
// time of an MMA here hardly shrinks with N (N = 192 measured no faster than
// 240), so the widest tile that TMEM holds twice issues the fewest MMAs.
//
// Epilogue.  TMEM lane 32 g + 8 j + t holds D[(j, 8 g + t)][.]: warp g reads
// its 32 lanes, each thread forms sum_i 160^i D (exact in int64), reduces it
// mod p and multiplies by 160^j mod p, and the 4 limbs of one output are
// added with two warp shuffles before the store.
//
// Work: tiles of 2048 outputs of every pair, taken by persistent CTAs (one
// per SM) from an atomic counter; the K-groups of a tile run one after the
// other on the CTA that took it.  Every wait on an mbarrier is bounded: when
// it runs out the kernel records PM_ERR_TIMEOUT and skips the remaining work.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "common.cuh"

namespace pm {

constexpr int TT = 32;                     // outputs per block
// Limb encoding (build-time choice): 1 = 4 balanced base-160 limbs of each operand (16
// limb products per modular MAC), 0 = 5 base-64 limbs of a x 4 base-256 limbs of b (20).
#ifndef PM_TC_ENC
#define PM_TC_ENC 1
#endif
#if PM_TC_ENC == 1
constexpr int NA_LIMB = 4, NB_LIMB = 4;
constexpr uint32_t BASE_A = 160, BASE_B = 160;
constexpr int TC_MAXK = 2592;   // terms per accumulated entry: 2592 * 80 * 80 = 16588800 <= 2^24
#else
constexpr int NA_LIMB = 5, NB_LIMB = 4;
constexpr uint32_t BASE_A = 64, BASE_B = 256;
constexpr int TC_MAXK = 4096;   // 4096 * 32 * 128 = 2^24
#endif
static_assert((int64_t)TC_MAXK * (BASE_A / 2) * (BASE_B / 2) <= (1 << 24), "fp32 sums stay exact");
static_assert(NB_LIMB == 4, "M = 128 rows: 4 limbs of b x 32 offsets");
#ifndef PM_TC_NBLK
#define PM_TC_NBLK (PM_TC_ENC == 1 ? 64 : 48)  // output blocks per tile (a multiple of 16)
#endif
constexpr int NBLK = PM_TC_NBLK;           // blocks per tile
constexpr int MMA_M = 128, MMA_N = NBLK * NA_LIMB;  // 256 (64 blocks x 4 limbs of a) or 240 (48 x 5)
static_assert(NBLK % 16 == 0 && MMA_N <= 256, "tile width");
constexpr int TILE_OUT = TT * NBLK;        // 2048 (or 1536)
constexpr int TC_GROUP = TC_MAXK / TT;     // shifts per K-group when both operands are longer
constexpr int64_t TC_MAX_DEG = PM_TENSOR_MAX_DEG;      // degrees this path takes (int tile indices)
constexpr int GROUP_D = 24;                // shifts per Hankel slot
constexpr int NH = 2;                      // Hankel slots in the ring
// (1024 pairs of degree 4095 / 64 of degree 16383, ms: 4 slots of 8 shifts 0.457 / 0.390, 6 of 8
// 0.461 / 0.394, 3 of 8 0.459 / 0.394, 2 of 16 0.431 / 0.365, 3 of 16 0.433 / 0.367, 2 of 24
// 0.425 / 0.369: fewer, larger slots mean fewer hand-overs between the builders and the MMAs)
constexpr int MAX_DELTA = TC_MAXK / TT + 2;            // shifts a tile can need
constexpr int BD_SHIFT = 7;                            // staged b digit t sits at index t + 7
constexpr int BD_LEN = TT * (MAX_DELTA + 2);           // b digits staged per limb (with the shift)
// limb stride in bf16 elements: an odd multiple of 8 words apart mod 32, so the 4 limbs sit on
// distinct bank groups
constexpr int BDS = BD_LEN + 2 * ((8 - (BD_LEN / 2) % 32 + 32) % 32);
constexpr int ROWS_MAX = NA_LIMB * (NBLK + MAX_DELTA + 2);
constexpr int B_LBO = ROWS_MAX * 16;                   // bytes between K chunks of the a operand
constexpr int B_BUF = 4 * B_LBO;                       // one a operand (double-buffered across tiles)
constexpr int H_Q = 4 * GROUP_D + 4;                   // Hankel core-matrix indices per slot (4 G + 3 used)
constexpr int H_SLOT = H_Q * 512;                      // 4 limbs x 128-byte core matrices per index
constexpr uint32_t TMEM_COLS = 512;                    // two accumulators of MMA_N columns
constexpr uint32_t ACC_STRIDE = 256;
constexpr int64_t WAIT_LIMIT = 1ll << 26;              // polls before a wait is declared lost (default)
static_assert((BDS / 2) % 32 == 8, "limb stride must spread the limbs over the banks");

// warp roles: 0 MMA issuer, 1-4 stagers (a operand), 5-12 builders (b digits,
// Hankel slots), 13-20 epilogue
// (measured on 1024 pairs of degree 4095, ms: builders 4 / 6 / 8 / 10 / 12 with 2 stagers
// 0.564 / 0.554 / 0.546 / 0.549 / 0.548; stagers 1 / 2 / 4 / 6 with 8 builders 0.597 / 0.545 /
// 0.537 / 0.535, 4 stagers with 10 builders 0.534)
constexpr int STG_WARP0 = 1, STG_WARPS = 4, STG_THREADS = 32 * STG_WARPS;
constexpr int BLD_WARP0 = STG_WARP0 + STG_WARPS, BLD_WARPS = 8, BLD_THREADS = 32 * BLD_WARPS;
constexpr int EPI_WARP0 = BLD_WARP0 + BLD_WARPS, EPI_WARPS = 8;
constexpr int TC_THREADS = 32 * (EPI_WARP0 + EPI_WARPS);  // 672

// shared memory map (bytes)
constexpr int SM_B = 0;                                   // 2 a operands: 4 chunks x ROWS_MAX rows each
constexpr int SM_H = SM_B + 2 * B_BUF;                    // ring of Hankel core-matrix slots
constexpr int SM_BD = SM_H + NH * H_SLOT;                 // b digits: NB_LIMB x BDS bf16
constexpr int SM_CTL = SM_BD + NB_LIMB * BDS * 2;         // mbarriers, tile records, TMEM address
constexpr int CTL_TILES = 256, CTL_EPI = 448, CTL_MISC = 512;
constexpr int TC_SMEM = SM_CTL + 576;

// mbarriers (index into the control block)
constexpr int BAR_A_FULL = 0;       // [2] tile record + a operand staged (stager leader)
constexpr int BAR_STAGE_EMPTY = 2;  // [2] MMAs of the tile that used the a operand done (commit)
constexpr int BAR_H_FULL = 4;       // [NH] Hankel slot built (builder leader)
constexpr int BAR_H_EMPTY = BAR_H_FULL + NH;      // [NH] MMAs reading the slot done (commit)
constexpr int BAR_ACC_FULL = BAR_H_EMPTY + NH;    // [2] accumulator complete: record written + MMAs done (2 arrivals)
constexpr int BAR_ACC_EMPTY = BAR_ACC_FULL + 2;   // [2] accumulator read back (one arrival per epilogue warp)
constexpr int BAR_DRAIN = BAR_ACC_EMPTY + 2;       // all MMAs issued by the CTA done
constexpr int NUM_BARS = BAR_DRAIN + 1;
static_assert(NUM_BARS * 8 <= CTL_TILES, "control block");

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

// instruction descriptor: D f32, A and B bf16, both K-major, N / 8 in bits 17-22, M / 16
// in bits 24-28 (every MMA spans the tile's full width: MMAs narrowed to the blocks a
// shift meets measured slower at every granularity)
constexpr uint32_t IDESC_BASE = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(MMA_M >> 4) << 24);
constexpr uint32_t IDESC = IDESC_BASE | ((uint32_t)(MMA_N >> 3) << 17);
static_assert(MMA_N % 16 == 0 && MMA_N <= 256, "MMA width");

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// plain arrival (release at CTA scope)
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar) : "memory");
}

// Bounded wait for phase `parity` of an mbarrier: at most `limit` polls; false
// if it ran out.
__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity, int64_t limit) {
    for (int64_t it = 0; it < limit; ++it) {
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

// Bounded wait by lane 0; once the phase has completed every lane waits on it
// too (returning at once), so that each reader acquires what was released
// before the arrival.  The result is the same on all lanes.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, int lane, int64_t limit) {
    int ok = 1;
    if (lane == 0) ok = wait_parity(bar, parity, limit);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) wait_parity(bar, parity, WAIT_LIMIT);  // completed: returns at the first poll
    return ok != 0;
}

// barriers among the stager warps and among the builder warps
__device__ __forceinline__ void stagers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(STG_THREADS) : "memory");
}
__device__ __forceinline__ void builders_sync() {
    asm volatile("bar.sync 2, %0;" ::"n"(BLD_THREADS) : "memory");
}

// Digit f - bias as an fp32 whose top half is its bf16 pattern (|f - bias| <= 128
// has at most 8 significant bits).  The word 0x4B400000 is 1.5 * 2^23, whose
// ulp is 1, so adding the integer f - bias to that word adds it to the value,
// and subtracting 1.5 * 2^23 leaves it exactly.
template <int BIAS>
__device__ __forceinline__ uint32_t digit_bits(uint32_t f) {
    return __float_as_uint(__uint_as_float(0x4B400000u - BIAS + f) - 12582912.0f);
}

// two bf16 in one word: x in the low half, y in the high half
__device__ __forceinline__ uint32_t pack2(uint32_t x, uint32_t y) {
    return __byte_perm(x, y, 0x7632);
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
    int n, m, L, I0, na, d_lo, d_hi, nd, J_min, nJ, tb0, done;
    int acc;   // a later K-group: add onto the residues already in c
};
static_assert(2 * sizeof(TcTile) <= CTL_EPI - CTL_TILES, "control block");

// what the epilogue needs of a tile
struct EpiInfo {
    uint32_t* c;
    int L, I0, done, acc;
};
static_assert(2 * sizeof(EpiInfo) <= CTL_MISC - CTL_EPI, "control block");

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
    tt.na = (tt.n + TT - 1) / TT;                       // blocks of a
    const int dmax = (tt.m + TT - 2) / TT;              // largest shift meeting b
    tt.d_lo = max(0, tt.I0 - tt.na + 1);
    tt.d_hi = min(dmax, tt.I0 + NBLK - 1);
    tt.nd = tt.d_hi - tt.d_lo + 1;                      // >= 1 for a tile inside [0, L)
    tt.J_min = tt.I0 - tt.d_hi;
    tt.nJ = NBLK + tt.d_hi - tt.d_lo;                   // blocks J_min .. J_min + nJ - 1
    tt.tb0 = TT * tt.d_lo - TT;                         // first staged b index
    tt.done = 0;
    tt.acc = 0;
    return tt;
}

// K-groups of a tile: one group when b (the shorter operand) has at most TC_MAXK
// terms, else groups of at most TC_GROUP shifts of about equal size.
__device__ __forceinline__ int tile_groups(const TcTile& t) {
    return t.m <= TC_MAXK ? 1 : (t.nd + TC_GROUP - 1) / TC_GROUP;
}

// Group g of ng of the tile: its shifts d_lo .. d_hi and the a blocks and b digits they use.
__device__ __forceinline__ TcTile sub_tile(const TcTile& t, int g, int ng) {
    TcTile u = t;
    const int gsz = (t.nd + ng - 1) / ng;
    u.d_lo = t.d_lo + g * gsz;
    u.d_hi = min(t.d_hi, u.d_lo + gsz - 1);
    u.nd = u.d_hi - u.d_lo + 1;
    u.J_min = u.I0 - u.d_hi;
    u.nJ = NBLK + u.d_hi - u.d_lo;
    u.tb0 = TT * u.d_lo - TT;
    u.acc = g > 0;
    return u;
}

struct TcParams {
    uint32_t p;
    uint64_t mu;             // floor(2^64 / p)
    uint64_t off;            // a multiple of p above 2^52 (makes signed limb sums non-negative)
    uint32_t wlo[NB_LIMB];   // BASE_B^j mod p
    uint32_t whi[NB_LIMB];   // 2^32 * BASE_B^j mod p
    int64_t wait_limit;      // polls before a wait between the roles is declared lost
};

// Balanced digits by an offset: with K = (B / 2) (1 + B + ... + B^(L-1)), u = v + K
// lies in [0, B^L) for |v| < p/2 < 2^28 (B = 160, L = 4: K = 329740880 and u in
// [61305424, 598176336]; B = 64, L = 5 and B = 256, L = 4 likewise), its standard
// base-B digits f_i give v = sum (f_i - B/2) B^i, the balanced digits in [-B/2, B/2).
template <uint32_t B, int L>
__host__ __device__ constexpr uint32_t digit_offset() {
    uint32_t k = 0, w = 1;
    for (int i = 0; i < L; ++i) {
        k += (B / 2) * w;
        w *= B;
    }
    return k;
}
constexpr uint32_t K_A = digit_offset<BASE_A, NA_LIMB>();
constexpr uint32_t K_B = digit_offset<BASE_B, NB_LIMB>();
template <uint32_t B, int L>
__host__ __device__ constexpr uint64_t digit_span() {  // B^L
    uint64_t w = 1;
    for (int i = 0; i < L; ++i) w *= B;
    return w;
}
static_assert(K_A >= (1u << 28) && (uint64_t)K_A + (1u << 28) <= digit_span<BASE_A, NA_LIMB>(), "digits of a");
static_assert(K_B >= (1u << 28) && (uint64_t)K_B + (1u << 28) <= digit_span<BASE_B, NB_LIMB>(), "digits of b");

// the next digit of u (u % B as bf16 bits of the balanced digit) and u / B
template <uint32_t B>
__device__ __forceinline__ uint32_t next_digit(uint32_t& u) {
    const uint32_t q = u / B, f = u - q * B;
    u = q;
    return digit_bits<B / 2>(f);
}

// a operand of a tile: row (NA_LIMB Jr + i) of K chunk kc holds limb i of
// a[32 (J_min + Jr) + 31 - 8 kc - e] at element e (K runs backwards).  One
// thread per block Jr: 32 coefficients, NA_LIMB limbs x 4 chunks of 16 bytes.
__device__ __forceinline__ void stage_a(const TcTile& tt, uint8_t* sBb, int stid, uint32_t p) {
    const int base = TT * tt.J_min;
    for (int Jr = stid; Jr < tt.nJ; Jr += STG_THREADS) {
        if (!PM_CHK(NA_LIMB * (Jr + 1) <= ROWS_MAX)) break;  // rows (NA_LIMB Jr + i) of every K chunk
        uint32_t u[TT];
#pragma unroll
        for (int k = 0; k < TT; ++k) {
            const int g = base + TT * Jr + k;
            u[k] = (g >= 0 && g < tt.n) ? (uint32_t)centred(__ldg(tt.a + g), p) + K_A : K_A;
        }
        uint8_t* dst = sBb + NA_LIMB * Jr * 16;
#pragma unroll
        for (int i = 0; i < NA_LIMB; ++i) {
            uint32_t f[TT];
#pragma unroll
            for (int k = 0; k < TT; ++k) f[k] = next_digit<BASE_A>(u[k]);
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {  // elements e = 0..7 are k = 31 - 8 kc - e
                const int k0 = 31 - 8 * kc;
                *reinterpret_cast<uint4*>(dst + kc * B_LBO + i * 16) =
                    make_uint4(pack2(f[k0], f[k0 - 1]), pack2(f[k0 - 2], f[k0 - 3]), pack2(f[k0 - 4], f[k0 - 5]),
                               pack2(f[k0 - 6], f[k0 - 7]));
            }
        }
    }
}

// b digits in natural order: position x of limb j holds d_j[tb0 + x - BD_SHIFT].
// One thread per 8 positions (positions 0..7 are never read), two groups of 8
// per pass so that their loads are in flight together.
__device__ __forceinline__ void stage_b_8(uint32_t (&u)[8], uint16_t* dst) {
#pragma unroll
    for (int j = 0; j < NB_LIMB; ++j) {
        uint32_t f[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) f[v] = next_digit<BASE_B>(u[v]);
        *reinterpret_cast<uint4*>(dst + j * BDS) =
            make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
}

__device__ __forceinline__ void stage_b(const TcTile& tt, uint16_t* sbd, int btid, uint32_t p) {
    const int nu = 4 * tt.nd + 5;  // positions up to 32 nd + 39, the last one a Hankel row reads
    if (!PM_CHK(8 * nu <= BD_LEN)) return;  // every staged position lies within a limb's array
    for (int u0 = 1 + btid; u0 < nu; u0 += 2 * BLD_THREADS) {
        const int u1 = u0 + BLD_THREADS;
        uint32_t x0[8], x1[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int g0 = tt.tb0 + 8 * u0 + v - BD_SHIFT, g1 = g0 + 8 * BLD_THREADS;
            x0[v] = (g0 >= 0 && g0 < tt.m) ? (uint32_t)centred(__ldg(tt.b + g0), p) + K_B : K_B;
            x1[v] = (u1 < nu && g1 >= 0 && g1 < tt.m) ? (uint32_t)centred(__ldg(tt.b + g1), p) + K_B : K_B;
        }
        stage_b_8(x0, sbd + 8 * u0);
        if (u1 < nu) stage_b_8(x1, sbd + 8 * u1);
    }
}

// Hankel core matrices H_j[q], q = 4 dg + qq: row t holds d_j[-31 + 8 q + t .. + 7].
// One thread per row; the 8 rows of one core matrix are 8 neighbouring
// threads writing 128 contiguous bytes.
__device__ __forceinline__ void build_hankel(const uint16_t* sbd, uint8_t* hslot, int nds, int dg, int tb0, int btid) {
    const uint32_t* sbw = reinterpret_cast<const uint32_t*>(sbd);
    const int nrow = (4 * nds + 3) * NB_LIMB * 8;
    const int ibase = BD_SHIFT - 31 + 32 * dg - tb0;  // staged index of d_j[-31 + 32 dg]: even
    if (!PM_CHK(nrow <= H_Q * NB_LIMB * 8 && ibase >= 0 && ibase + 8 * (4 * nds + 3) + 10 <= BD_LEN)) return;
    for (int rw = btid; rw < nrow; rw += BLD_THREADS) {
        const int t = rw & 7, j = (rw >> 3) & 3, qq = rw >> 5;
        const int e0 = j * BDS + ibase + 8 * qq + t;
        const uint32_t* wp = sbw + (e0 >> 1);
        const uint32_t sh = (uint32_t)(t & 1) * 16;
        const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2], w3 = wp[3], w4 = wp[4];
        *reinterpret_cast<uint4*>(hslot + qq * 512 + j * 128 + t * 16) =
            make_uint4(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh), __funnelshift_r(w2, w3, sh),
                       __funnelshift_r(w3, w4, sh));
    }
}

// Warp-specialised persistent kernel.  Warp 0 issues the MMAs (one thread)
// into two TMEM accumulators used by alternate tiles; warps 1-4 claim tiles and
// stage the a operand (double-buffered, so the next tile's is ready before the
// current one's MMAs end); warps 5-12 stage the b digits of a tile and build its
// Hankel slots ahead of the MMAs; warps 13-20 read an accumulator back and
// reduce it while the next tile accumulates into the other one.  The roles
// hand over through mbarriers only.
__global__ void __launch_bounds__(TC_THREADS, 1) tc_batched_kernel(
    int batch, const uint32_t* __restrict__ a_data, const int64_t* __restrict__ a_off,
    const uint32_t* __restrict__ b_data, const int64_t* __restrict__ b_off,
    uint32_t* __restrict__ c_data, const int64_t* __restrict__ c_off, const int64_t* __restrict__ prefix,
    unsigned long long* __restrict__ counter, TcParams tp, int* status) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint16_t* sbd = reinterpret_cast<uint16_t*>(sm + SM_BD);
    TcTile* s_tiles = reinterpret_cast<TcTile*>(sm + SM_CTL + CTL_TILES);
    EpiInfo* s_epi = reinterpret_cast<EpiInfo*>(sm + SM_CTL + CTL_EPI);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + SM_CTL + CTL_MISC);
    volatile int* s_abort = reinterpret_cast<volatile int*>(sm + SM_CTL + CTL_MISC + 4);
    volatile int* s_pstop = reinterpret_cast<volatile int*>(sm + SM_CTL + CTL_MISC + 8);
    volatile int* s_sstop = reinterpret_cast<volatile int*>(sm + SM_CTL + CTL_MISC + 12);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar0 = smem_u32(sm + SM_CTL);
    auto bar = [bar0](int i) { return bar0 + 8u * (uint32_t)i; };
    auto fail = [status, s_abort]() {
        atomicCAS(status, 0, (int)PM_ERR_TIMEOUT);
        *s_abort = 1;
    };

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar(BAR_A_FULL + i), 1);
            mbar_init(bar(BAR_STAGE_EMPTY + i), 1);
            mbar_init(bar(BAR_ACC_FULL + i), 2);
            mbar_init(bar(BAR_ACC_EMPTY + i), EPI_WARPS);
        }
        for (int i = 0; i < NH; ++i) {
            mbar_init(bar(BAR_H_FULL + i), 1);
            mbar_init(bar(BAR_H_EMPTY + i), 1);
        }
        mbar_init(bar(BAR_DRAIN), 1);
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
    pdl_wait();  // the planner's prefix and counter (nothing above touches global memory)
    const int64_t total = prefix[batch];
    const int64_t WL = tp.wait_limit;

    if (warp == 0) {
        // ---------------- MMA issuer ----------------
        uint32_t G = 0;  // Hankel groups consumed
        for (int k = 0;; ++k) {
            const int sb = k & 1;
            int ok = warp_wait(bar(BAR_A_FULL + sb), (k >> 1) & 1, lane, WL);
            if (ok && k >= 2) ok = warp_wait(bar(BAR_ACC_EMPTY + sb), ((k >> 1) - 1) & 1, lane, WL);
            if (!ok) {
                if (lane == 0) fail();
                break;
            }
            const TcTile tt = s_tiles[sb];
            if (lane == 0) {
                s_epi[sb] = EpiInfo{tt.c, tt.L, tt.I0, tt.done, tt.acc};
                mbar_arrive(bar(BAR_ACC_FULL + sb));  // the record (the second arrival is the MMAs')
                if (tt.done) mbar_arrive(bar(BAR_ACC_FULL + sb));
            }
            if (tt.done) break;
            const uint32_t tacc = tmem + (uint32_t)sb * ACC_STRIDE;
            const uint32_t sBa = smem_u32(sm + SM_B + sb * B_BUF);
            const int ngroups = (tt.nd + GROUP_D - 1) / GROUP_D;
            for (int gi = 0; gi < ngroups && ok; ++gi, ++G) {
                const int slot = (int)(G % NH);
                if (lane == 0) {
                    ok = wait_parity(bar(BAR_H_FULL + slot), (G / NH) & 1, WL);
                    if (!ok) {
                        fail();
                    } else {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t ha = smem_u32(sm + SM_H + slot * H_SLOT);
                        const int nds = min(GROUP_D, tt.nd - gi * GROUP_D);
                        const int dg = tt.d_lo + gi * GROUP_D;
                        for (int s = 0; s < nds; ++s) {
                            const bool first = gi == 0 && s == 0;
                            // a's rows of this shift and the slot's core matrices (16 row groups of
                            // 128 bytes from the shift's K offset, two K chunks 512 bytes apart) lie
                            // in their buffers
                            if (!PM_CHK(NA_LIMB * (tt.d_hi - dg - s) + MMA_N <= ROWS_MAX &&
                                        tt.d_hi - dg - s >= 0 && (4 * s + 7) * 512 <= H_SLOT))
                                continue;
                            const uint32_t b_addr = sBa + (uint32_t)(NA_LIMB * (tt.d_hi - dg - s) * 16);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const uint64_t da = smem_desc(ha + (uint32_t)((4 * s + 2 * h) * 512), 512, 128);
                                const uint64_t db = smem_desc(b_addr + 2 * h * B_LBO, B_LBO, 128);
                                mma_bf16(tacc, da, db, IDESC, (first && h == 0) ? 0u : 1u);
                            }
                        }
                        mma_commit(bar(BAR_H_EMPTY + slot));
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
            }
            if (!ok) break;
            if (lane == 0) {
                mma_commit(bar(BAR_STAGE_EMPTY + sb));
                mma_commit(bar(BAR_ACC_FULL + sb));
            }
            __syncwarp();
        }
        if (lane == 0) {  // every MMA of this CTA completes before TMEM is released
            // (with the built-in limit whatever the roles' limit is: the MMAs issued so
            // far always complete, and TMEM must not be freed under them)
            mma_commit(bar(BAR_DRAIN));
            if (!wait_parity(bar(BAR_DRAIN), 0, WAIT_LIMIT)) fail();
        }
        __syncwarp();
    } else if (warp < BLD_WARP0) {
        // ---------------- stagers: claim tiles, a operand ----------------
        // The record s_tiles[sb] is rewritten only once the MMAs of the tile that
        // used it are complete (STAGE_EMPTY), when every reader has its copy.  A
        // stager that stops (a wait ran out, or another role failed) writes no
        // record and arrives at nothing: the other roles then end through their
        // own bounded waits, and no reader can see a record being rewritten.
        // Each claimed tile is handed on as its K-groups, one record per group.
        const int stid = tid - 32 * STG_WARP0;
        TcTile cur{};       // the claimed tile (stid 0 only)
        int g = 0, ng = 0;  // its next group and number of groups
        for (int k = 0;; ++k) {
            const int sb = k & 1;
            if (stid == 0) {
                bool stop = *s_abort != 0;
                if (!stop && k >= 2 && !wait_parity(bar(BAR_STAGE_EMPTY + sb), ((k >> 1) - 1) & 1, WL)) {
                    fail();
                    stop = true;
                }
                if (!stop) {
                    TcTile tt{};
                    if (g >= ng) {  // claim the next tile
                        const int64_t tile = (int64_t)atomicAdd(counter, 1ull);
                        if (tile < total) {
                            cur = make_tile(tile, batch, a_data, a_off, b_data, b_off, c_data, c_off, prefix);
                            g = 0;
                            ng = tile_groups(cur);
                        } else {
                            tt.done = 1;
                        }
                    }
                    if (!tt.done) tt = sub_tile(cur, g++, ng);
                    s_tiles[sb] = tt;
                }
                *s_sstop = stop;
            }
            stagers_sync();
            if (*s_sstop) break;  // (read by every stager before stid 0 can write it again)
            const TcTile tt = s_tiles[sb];
            if (!tt.done) {
                stage_a(tt, sm + SM_B + sb * B_BUF, stid, tp.p);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                stagers_sync();
            }
            if (stid == 0) mbar_arrive(bar(BAR_A_FULL + sb));
            if (tt.done) break;
        }
    } else if (warp < EPI_WARP0) {
        // ---------------- builders: b digits, Hankel slots ----------------
        const int btid = tid - 32 * BLD_WARP0;
        uint32_t G = 0;  // Hankel groups built
        for (int k = 0;; ++k) {
            const int sb = k & 1;
            if (btid == 0) {
                bool stop = *s_abort != 0;
                if (!stop && !wait_parity(bar(BAR_A_FULL + sb), (k >> 1) & 1, WL)) {
                    fail();
                    stop = true;
                }
                *s_pstop = stop;
            }
            builders_sync();
            if (*s_pstop) break;
            wait_parity(bar(BAR_A_FULL + sb), (k >> 1) & 1, WAIT_LIMIT);  // completed: acquires the tile record
            const TcTile tt = s_tiles[sb];
            if (tt.done) break;
            // the whole tile's b digits at once: their loads are all in flight together, and the
            // MMAs of the previous tile's last slots (up to NH of them) cover the time
            stage_b(tt, sbd, btid, tp.p);
            const int ngroups = (tt.nd + GROUP_D - 1) / GROUP_D;
            bool stop = false;
            for (int gi = 0; gi < ngroups; ++gi, ++G) {
                const int slot = (int)(G % NH);
                builders_sync();  // (the b digits are complete before the first slot)
                if (btid == 0) {
                    bool st = *s_abort != 0;
                    if (!st && G >= NH && !wait_parity(bar(BAR_H_EMPTY + slot), ((G / NH) - 1) & 1, WL)) {
                        fail();
                        st = true;
                    }
                    *s_pstop = st;
                }
                builders_sync();
                if (*s_pstop) {
                    stop = true;
                    break;
                }
                build_hankel(sbd, sm + SM_H + slot * H_SLOT, min(GROUP_D, tt.nd - gi * GROUP_D),
                             tt.d_lo + gi * GROUP_D, tt.tb0, btid);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                builders_sync();
                if (btid == 0) mbar_arrive(bar(BAR_H_FULL + slot));
            }
            if (stop) break;
            builders_sync();  // every builder is past the last slot before the b digits change
        }
    } else {
        // ---------------- epilogue ----------------
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 = (limb j, offset 8 (w % 4) + t) and
        // half of the columns (NBLK / 2 blocks); the 4 limbs of an output sit on lanes t, t + 8,
        // t + 16, t + 24 and are combined by a reduce-scatter over 4 blocks at a time.
        const int quarter = warp & 3, half = (warp - EPI_WARP0) >> 2;
        const int j = lane >> 3, r = 8 * quarter + (lane & 7);
        // (constant indices: a dynamic index would copy the parameters to local memory)
        const uint32_t wlo = j == 0 ? tp.wlo[0] : j == 1 ? tp.wlo[1] : j == 2 ? tp.wlo[2] : tp.wlo[3];
        const uint32_t whi = j == 0 ? tp.whi[0] : j == 1 ? tp.whi[1] : j == 2 ? tp.whi[2] : tp.whi[3];
        for (int k = 0;; ++k) {
            const int ab = k & 1;
            if (!warp_wait(bar(BAR_ACC_FULL + ab), (k >> 1) & 1, lane, WL)) {
                if (lane == 0) fail();
                break;
            }
            const EpiInfo info = s_epi[ab];
            if (info.done) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t tbase = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)ab * ACC_STRIDE +
                                   (uint32_t)(half * (MMA_N / 2));
#pragma unroll 1
            for (int rd = 0; rd < NBLK / 16; ++rd) {  // 8 blocks (8 NA_LIMB columns) per round
                uint32_t v[8 * NA_LIMB];
#pragma unroll
                for (int q = 0; q < NA_LIMB; ++q) {
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                        : "=r"(v[8 * q + 0]), "=r"(v[8 * q + 1]), "=r"(v[8 * q + 2]), "=r"(v[8 * q + 3]),
                          "=r"(v[8 * q + 4]), "=r"(v[8 * q + 5]), "=r"(v[8 * q + 6]), "=r"(v[8 * q + 7])
                        : "r"(tbase + (uint32_t)(8 * NA_LIMB * rd + 8 * q)));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (rd == NBLK / 16 - 1) {  // the accumulator is free once its last columns are in registers
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(BAR_ACC_EMPTY + ab));
                }
#pragma unroll
                for (int c4 = 0; c4 < 2; ++c4) {
                    uint64_t x[4];
#pragma unroll
                    for (int be = 0; be < 4; ++be) {
                        const uint32_t* dv = v + NA_LIMB * (4 * c4 + be);
                        // off + sum_i BASE_A^i d_i with |d_i| <= 2^24: |sum| < 2^49, so u lies in [0, 2^53)
                        int64_t sum = (int64_t)tp.off;
                        int64_t wa = 1;
#pragma unroll
                        for (int i = 0; i < NA_LIMB; ++i) {
                            sum += (int64_t)__float2int_rn(__uint_as_float(dv[i])) * wa;
                            wa *= BASE_A;
                        }
                        const uint64_t u = (uint64_t)sum;
                        x[be] = (uint64_t)(uint32_t)u * wlo + (uint64_t)(uint32_t)(u >> 32) * whi;  // < 2^61.01
                    }
                    // reduce-scatter over the limbs: lane (j, t) ends with block 4 c4 + j
                    const bool o1 = (j & 1) != 0;
                    const uint64_t keep0 = o1 ? x[1] : x[0], send0 = o1 ? x[0] : x[1];
                    const uint64_t keep1 = o1 ? x[3] : x[2], send1 = o1 ? x[2] : x[3];
                    const uint64_t y0 = keep0 + __shfl_xor_sync(0xffffffffu, send0, 8);
                    const uint64_t y1 = keep1 + __shfl_xor_sync(0xffffffffu, send1, 8);
                    const bool o2 = (j & 2) != 0;
                    const uint64_t z = (o2 ? y1 : y0) + __shfl_xor_sync(0xffffffffu, o2 ? y0 : y1, 16);  // < 2^64
                    const int blk = NBLK / 2 * half + 8 * rd + 4 * c4 + j;
                    const int g = (info.I0 + blk) * TT + r;
                    if (g < info.L) {
                        // a later K-group adds onto the residue this thread wrote for the earlier
                        // groups (same thread, same word: program order); z < 2^63.01
                        const uint64_t prev = info.acc ? (uint64_t)info.c[g] : 0ull;
                        info.c[g] = barrett(z + prev, tp.p, tp.mu);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// Planner: validates the CSR layout (degrees <= max_deg <= 4095) and builds
// the prefix of tile counts; resets the tile counter.
__global__ void __launch_bounds__(1024) tc_plan_kernel(int batch, const int64_t* __restrict__ a_off,
                                                        const int64_t* __restrict__ b_off,
                                                        const int64_t* __restrict__ c_off, int64_t max_deg,
                                                        int64_t min_short, int64_t* prefix,
                                                        unsigned long long* counter, int* status) {
    __shared__ long long s_scan[1024];
    __shared__ int s_bad;
    pdl_trigger();  // the product kernel may be placed now; it waits for this one to end
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
        run += min(n, m) >= min_short ? (n + m - 1 + TILE_OUT - 1) / TILE_OUT : 0;
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
        pos += min(n, m) >= min_short ? (n + m - 1 + TILE_OUT - 1) / TILE_OUT : 0;
    }
    if (tid == 1023) {
        prefix[batch] = s_scan[1023];
        *counter = 0;
    }
}

// ---- Measurement: the rate and the exactness of one tcgen05 MMA kind ----
// kind 0: kind::f16 with bf16 operands (K = 16 per MMA, the product kernel's
// kind); kind 1: kind::f8f6f4 with e4m3 operands (K = 32), the 8-bit limb
// encoding's.  Every operand is a constant, so the result does not depend on
// the core-matrix layout: A holds `big` (bf16 128 or e4m3 16) or 1, B holds 1.
// Exactness: r_big MMAs of the big A and then r_small of A = 1 accumulate
// r_big K big + r_small K, an integer below 2^24 that fp32 holds exactly, into
// every accumulator entry; the small addends land on a sum near 2^23, so an
// accumulation that kept fewer bits than fp32 would drop them.  Rate: r_rate
// further full-width MMAs (M = 128, N = 256) issued back to back by one
// thread, timed on the SM's cycle counter from the first issue to their
// completion (commit and wait).  Each wait is bounded.
constexpr int MP_THREADS = 128, MP_N = 256;
constexpr int MP_A_BYTES = 128 * 32, MP_B_BYTES = MP_N * 32;  // rows x 32 bytes of K
constexpr int MP_SMEM = 2 * MP_A_BYTES + MP_B_BYTES + 64;

struct MmaProbeRec {
    long long start, end;
    uint32_t value, mismatches;
    int smid, status;
};

__device__ __forceinline__ void mma_probe_issue(int kind, uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                                uint32_t acc) {
    if (kind == 0) {
        mma_bf16(tmem, da, db, idesc, acc);
    } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
}

__global__ void __launch_bounds__(MP_THREADS, 1) tc_mma_probe_kernel(int kind, int r_big, int r_small, int r_rate,
                                                                      uint32_t expect_bits,
                                                                      MmaProbeRec* __restrict__ rec) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t* a_big = sm;
    uint8_t* a_one = sm + MP_A_BYTES;
    uint8_t* b_one = sm + 2 * MP_A_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * MP_A_BYTES + MP_B_BYTES);  // [0] phases, [1] drain
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2);
    int* s_status = reinterpret_cast<int*>(bars + 3);
    uint32_t* s_bad = reinterpret_cast<uint32_t*>(bars + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t w_big = kind ? 0x58585858u : 0x43004300u;  // e4m3 16.0 / bf16 128.0
    const uint32_t w_one = kind ? 0x38383838u : 0x3F803F80u;  // e4m3 1.0 / bf16 1.0
    for (int i = tid; i < MP_A_BYTES / 4; i += MP_THREADS) {
        reinterpret_cast<uint32_t*>(a_big)[i] = w_big;
        reinterpret_cast<uint32_t*>(a_one)[i] = w_one;
    }
    for (int i = tid; i < MP_B_BYTES / 4; i += MP_THREADS) reinterpret_cast<uint32_t*>(b_one)[i] = w_one;
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_status = 0;
        *s_bad = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // operands visible to the tensor core
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(MP_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *s_tmem;
    const uint32_t idesc = (1u << 4) | (kind ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(MP_N >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    const uint64_t da_big = smem_desc(smem_u32(a_big), 128, 256);
    const uint64_t da_one = smem_desc(smem_u32(a_one), 128, 256);
    const uint64_t db = smem_desc(smem_u32(b_one), 128, 256);
    if (tid == 0) {
        for (int i = 0; i < r_big; ++i) mma_probe_issue(kind, tmem, da_big, db, idesc, i > 0 ? 1u : 0u);
        for (int i = 0; i < r_small; ++i) mma_probe_issue(kind, tmem, da_one, db, idesc, 1u);
        mma_commit(smem_u32(&bars[0]));
        if (!wait_parity(smem_u32(&bars[0]), 0, WAIT_LIMIT)) *s_status = PM_ERR_TIMEOUT;
    }
    __syncthreads();
    if (*s_status == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // each warp reads its 32 lanes at 4 columns spread over the accumulator
        uint32_t v[4];
        const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                         : "=r"(v[q])
                         : "r"(base + (uint32_t)(q * (MP_N / 4) + 17 * q)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        uint32_t bad = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) bad += v[q] != expect_bits;
        if (bad) atomicAdd(s_bad, bad);
        if (tid == 0) rec[blockIdx.x].value = v[0];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        long long t0 = clock64(), t1 = t0;
        if (*s_status == 0) {
            for (int i = 0; i < r_rate; ++i) mma_probe_issue(kind, tmem, da_big, db, idesc, i > 0 ? 1u : 0u);
            mma_commit(smem_u32(&bars[0]));
            if (!wait_parity(smem_u32(&bars[0]), 1, WAIT_LIMIT)) *s_status = PM_ERR_TIMEOUT;
            t1 = clock64();
        }
        // every MMA this thread issued is complete before the tensor memory is freed
        mma_commit(smem_u32(&bars[1]));
        if (!wait_parity(smem_u32(&bars[1]), 0, WAIT_LIMIT)) *s_status = PM_ERR_TIMEOUT;
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        rec[blockIdx.x].start = t0;
        rec[blockIdx.x].end = t1;
        rec[blockIdx.x].smid = (int)smid;
        rec[blockIdx.x].status = *s_status;
        rec[blockIdx.x].mismatches = *s_bad;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MP_N));
    }
}

pm_status launch_mma_probe(int kind, int64_t iters, double* flops_per_clk_sm, int* exact, cudaStream_t st,
                           DeviceWorkspace* ws) {
    if (ws->cc_major != 10) return PM_ERR_UNSUPPORTED;  // tcgen05 needs the sm_100 family
    const int nblk = ws->num_sms;
    const int K = kind ? 32 : 16, big = kind ? 16 : 128;
    // r_big MMAs bring the sum near 2^23; r_small addends follow (exact integers below 2^24)
    const int r_big = (int)(((1 << 23) - 1) / ((int64_t)K * big)), r_small = 300;
    const float expect = (float)((int64_t)r_big * K * big + (int64_t)r_small * K);
    uint32_t expect_bits;
    memcpy(&expect_bits, &expect, sizeof(expect_bits));
    MmaProbeRec* d_rec = nullptr;
    if (dev_alloc((void**)&d_rec, sizeof(MmaProbeRec) * (size_t)nblk) != cudaSuccess) {
        cudaGetLastError();
        return PM_ERR_NOMEM;
    }
    std::vector<MmaProbeRec> h((size_t)nblk);
    cudaError_t e = cudaFuncSetAttribute(tc_mma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MP_SMEM);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_rec, 0, sizeof(MmaProbeRec) * (size_t)nblk, st);
    if (e == cudaSuccess) {
        tc_mma_probe_kernel<<<nblk, MP_THREADS, MP_SMEM, st>>>(kind, r_big, r_small, (int)iters, expect_bits, d_rec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_rec, sizeof(MmaProbeRec) * (size_t)nblk, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_rec);
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(1);
    // per SM: the MMAs of its blocks over the cycles from its first start to its last end
    std::map<int, std::pair<long long, long long>> span;
    std::map<int, int> cnt;
    int ok = 1;
    for (const MmaProbeRec& r : h) {
        if (r.status != 0) return (pm_status)r.status;
        if (r.mismatches != 0 || r.value != expect_bits) ok = 0;
        auto it = span.find(r.smid);
        if (it == span.end()) {
            span[r.smid] = {r.start, r.end};
        } else {
            it->second.first = std::min(it->second.first, r.start);
            it->second.second = std::max(it->second.second, r.end);
        }
        ++cnt[r.smid];
    }
    const double flops = 2.0 * 128 * MP_N * K * (double)iters;
    double sum = 0.0;
    int used = 0;
    for (const auto& kv : span) {
        const long long c = kv.second.second - kv.second.first;
        if (c <= 0) continue;
        sum += flops * cnt[kv.first] / (double)c;
        ++used;
    }
    if (!used) return PM_ERR_INTERNAL;
    *flops_per_clk_sm = sum / used;
    *exact = ok;
    return PM_OK;
}

pm_status launch_batched_tensor(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                                const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                                const int64_t* c_off, uint32_t p, int64_t max_deg, int64_t min_short,
                                cudaStream_t st, DeviceWorkspace* ws) {
    if (p >= (1u << 29) || max_deg > TC_MAX_DEG) return PM_ERR_UNSUPPORTED;
    if (ws->cc_major != 10) return PM_ERR_UNSUPPORTED;  // tcgen05 needs the sm_100 family
    StreamScratch* sc = nullptr;
    pm_status rc = stream_scratch(ws, st, &sc);
    if (rc != PM_OK) return rc;
    rc = ensure_scratch(&sc->tc, &sc->tc_bytes, 256 + sizeof(int64_t) * (size_t)(batch + 1), st, false);
    if (rc != PM_OK) return rc;
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(sc->tc);
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
    const int64_t wl = tc_wait_limit();
    tp.wait_limit = wl > 0 ? wl : WAIT_LIMIT;
    uint64_t w = 1;
    for (int j = 0; j < NB_LIMB; ++j) {
        tp.wlo[j] = (uint32_t)w;
        tp.whi[j] = (uint32_t)((w << 32) % p);
        w = (w * BASE_B) % p;
    }
    e = chk_bind(ws);
    if (e != cudaSuccess) return cuda_fail(e);
    tc_plan_kernel<<<1, 1024, 0, st>>>((int)batch, a_off, b_off, c_off, max_deg, min_short, prefix, counter,
                                       ws->status);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_dep(tc_batched_kernel, dim3(ws->num_sms), dim3(TC_THREADS), TC_SMEM, st, (int)batch, a_data,
                       a_off, b_data, b_off, c_data, c_off, (const int64_t*)prefix, counter, tp, ws->status);
    if (e != cudaSuccess) return cuda_fail(e);
    count_launches(2);
    return PM_OK;
}

}  // namespace pm

extern "C" pm_status polymul_tensor_limbs(int* na, int* nb, uint32_t* base_a, uint32_t* base_b, int* max_terms,
                                          int* tile_blocks) {
    if (!na || !nb || !base_a || !base_b || !max_terms || !tile_blocks) return PM_ERR_INVALID_ARG;
    *tile_blocks = pm::NBLK;
    *na = pm::NA_LIMB;
    *nb = pm::NB_LIMB;
    *base_a = pm::BASE_A;
    *base_b = pm::BASE_B;
    *max_terms = pm::TC_MAXK;
    return PM_OK;
}
