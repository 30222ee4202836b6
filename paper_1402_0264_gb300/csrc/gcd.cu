// Greatest common divisor over Z/pZ, p prime (Section 6, "The Euclidean
// algorithm for polynomials"): the monic gcd of a and b.
//
// Paper -> this file.  Algorithms 8-9 (the naive gcd) run one division step
// per kernel call: the polynomial of larger degree (a when the degrees are
// equal) loses its leading term to a multiple of the other, the degree of
// the reduced one is lowered past any new zero leading coefficients, and the
// calls stop once one polynomial is zero or constant.  Algorithms 10-11 run s
// such steps per call: every thread-block copies the s-heads (leading
// coefficients) of both polynomials, runs the s steps on them to learn the
// leading coefficients each step needs, and updates its own stretch of a and
// b, with a window of 2s coefficients around it since consecutive blocks
// share s coefficients.  Here each launch of gcd_round_kernel is one such
// call:
//   head: warp 0 runs up to s steps on heads of H = s + 32 leading
//         coefficients of each polynomial and records each step (which
//         polynomial is reduced, the two multipliers, the relative shift);
//         it tracks how far each head is still exact (a step on a can only
//         update the entries of a's head whose partner in b's head is known)
//         and ends the round early when a leading coefficient it needs is
//         past that point (the next round reloads the heads);
//   body: every block then replays the recorded steps, in order, on a window
//         of both polynomials around its T positions, with a halo on each
//         side as wide as the largest degree drop of the round (no value of
//         an output position depends on anything farther away), and writes
//         its T positions to the other copy of the arrays.
// Steps are fraction-free: reducing a by b is a <- lc(b) a - lc(a) x^d b
// (and the same with a and b exchanged), which cancels the leading term like
// the paper's a - lc(a) lc(b)^-1 x^d b but is a unit multiple of it, so the
// sequence of degrees and the gcd up to a unit are the same, and no modular
// inverse sits on the sequential path; one inverse at the end makes the
// result monic.  For odd p each step's words are reduced by Montgomery's
// method (P. Montgomery, "Modular multiplication without trial division",
// Math. Comp. 1985) without converting to Montgomery form, which scales the
// step by the unit 2^-32 mod p and leaves degrees and the gcd unchanged.  A polynomial that becomes a nonzero constant ends the
// computation with gcd 1 (the paper's test "zero or constant" would return
// the other polynomial there).
//
// The number of steps is at most deg a + deg b + 2 and is data dependent,
// so the host launches rounds in batches and reads the state back between
// batches (the call synchronises its stream).
#include <algorithm>

#include "common.cuh"

namespace pm {

// (degrees 9999 and 8999, s = 64, ms: 256 positions and 512 threads per block 9.51, 128 and 512
// 9.37, 64 and 512 10.02, 256 and 256 10.52, 128 and 256 9.19, 64 and 256 9.32, 128 and 128 10.58)
constexpr int GCD_THREADS = 256;               // 8 warps
constexpr int GCD_T = 128;                     // output positions per block
constexpr int GCD_SMAX = 256;                  // largest s
constexpr int GCD_HEXTRA = 32;                 // head length H = s + GCD_HEXTRA
constexpr int GCD_HMAX = GCD_SMAX + GCD_HEXTRA;
constexpr int GCD_WMAX = GCD_T + 2 * GCD_HMAX; // window words per polynomial
constexpr int GCD_J = (GCD_WMAX + GCD_THREADS - 1) / GCD_THREADS;  // window words per thread

enum GcdKind : int { GCD_IS_A = 0, GCD_IS_B = 1, GCD_IS_ONE = 2, GCD_IS_ZERO = 3 };

// State between rounds (two copies, alternating: a round reads one and
// writes the other, so no block of a round sees its own round's update).
struct GcdState {
    int64_t da, db;   // degree bounds of a and b (leading coefficients may still be zero)
    int64_t dg;       // degree of the gcd once done (-1: both zero)
    int32_t done;     // 1 once the gcd is known
    int32_t kind;     // GcdKind
    int32_t buf;      // copy (0/1) of the arrays that holds the final a and b
    int32_t steps_lo; // division steps so far (low 32 bits, diagnostic)
    int64_t rounds;   // rounds that did work
};
static_assert(sizeof(GcdState) == 48, "GcdState layout");

struct GcdMod {
    uint32_t p;
    uint32_t pinv;   // -p^-1 mod 2^32 (odd p)
    uint64_t mu;     // floor(2^64 / p)
};

// For x, y, c1, c2n < p < 2^30: MONT (odd p) gives (c1 x + c2n y) 2^-32 mod p
// (v = c1 x + c2n y < 2p^2; q = v (-p^-1) mod 2^32 makes v + q p a multiple of
// 2^32, and (v + q p) / 2^32 < 2p^2 / 2^32 + p < 2p); otherwise
// (c1 x + c2n y) mod p by Barrett's method.
template <bool MONT>
__device__ __forceinline__ uint32_t gcd_comb(uint32_t c1, uint32_t x, uint32_t c2n, uint32_t y, const GcdMod& m) {
    const uint64_t v = (uint64_t)c1 * x + (uint64_t)c2n * y;
    if (MONT) {
        const uint32_t q = (uint32_t)v * m.pinv;
        const uint32_t r = (uint32_t)((v + (uint64_t)q * m.p) >> 32);
        return r >= m.p ? r - m.p : r;
    }
    return barrett(v, m.p, m.mu);
}

// Copies a and b reduced mod p into the first copy of the arrays and writes
// the initial state.
__global__ void gcd_init_kernel(const uint32_t* __restrict__ a, int64_t na, const uint32_t* __restrict__ b,
                                int64_t nb, uint32_t* __restrict__ A0, uint32_t* __restrict__ B0, uint32_t p,
                                GcdState* st) {
    pdl_trigger();  // the first round may be placed now; it waits for this kernel to end
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < na; x += stride) A0[x] = a[x] % p;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nb; x += stride) B0[x] = b[x] % p;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        GcdState s0{};
        s0.da = na - 1;
        s0.db = nb - 1;
        s0.dg = -1;
        st[0] = s0;
        st[1] = s0;
    }
}

// Lowers u (offset of the leading coefficient from the round's top) past
// zero head entries, one warp-wide ballot per 32 entries.  lim = first offset
// that is not a known coefficient (the head's exact length, or one past the
// constant term).  Returns the leading coefficient when found (u < lim).
__device__ __forceinline__ uint32_t gcd_strip(const uint32_t* h, int& u, int lim, int lane) {
    for (int guard = 0; guard < GCD_HMAX / 32 + 2; ++guard) {
        if (u >= lim) return 0;
        const int idx = u + lane;
        const uint32_t v = idx < lim ? h[idx] : 0u;
        const unsigned msk = __ballot_sync(0xffffffffu, v != 0u);
        if (msk) {
            const int f = __ffs(msk) - 1;
            u += f;
            return __shfl_sync(0xffffffffu, v, f);
        }
        u = min(u + 32, lim);
    }
    return 0;
}

// One round.  X* are the arrays at the round's start, Y* receive the result;
// sin/sout the state copies; ybuf names Y's copy for the final state.
template <bool MONT>
__global__ void __launch_bounds__(GCD_THREADS, 1) gcd_round_kernel(
    const uint32_t* __restrict__ XA, const uint32_t* __restrict__ XB, uint32_t* __restrict__ YA,
    uint32_t* __restrict__ YB, const GcdState* __restrict__ sin, GcdState* __restrict__ sout, int s, int H,
    int ybuf, GcdMod md) {
    const uint32_t p = md.p;
    __shared__ uint32_t hAB[2 * GCD_HMAX];   // heads: a at [0, GCD_HMAX), b at [GCD_HMAX, 2 GCD_HMAX)
    __shared__ uint32_t rc1[GCD_SMAX], rc2[GCD_SMAX];
    __shared__ int rsig[GCD_SMAX];       // (shift << 1) | (1 when b is the reduced one)
    __shared__ uint32_t wA[GCD_WMAX], wB[GCD_WMAX];
    __shared__ int r_k, r_ua, r_ub, r_kind;
    __shared__ int64_t r_dg;

    // (uniform: before any barrier) the heads, step records and windows fit their arrays
    if (!PM_CHK(H <= GCD_HMAX && s <= GCD_SMAX && GCD_T + 2 * H <= GCD_WMAX && blockDim.x == GCD_THREADS)) return;
    pdl_wait();  // the previous round's arrays and state
    pdl_trigger();
    const GcdState s0 = *sin;
    const int tid = threadIdx.x;
    if (s0.done) {
        if (blockIdx.x == 0 && tid == 0) *sout = s0;
        return;
    }
    const int64_t da0 = s0.da, db0 = s0.db;
    const int64_t i0 = (int64_t)blockIdx.x * GCD_T;   // first offset (from the round's tops) of this block
    if (i0 > max(da0, db0) && blockIdx.x != 0) return;
    const int Wn = GCD_T + 2 * H;

    if (tid >= 32) {
        // window: offsets i0 - H .. i0 + T + H - 1 of both polynomials (zero above the top and below x^0)
        for (int t = tid - 32; t < Wn; t += GCD_THREADS - 32) {
            const int64_t i = i0 - H + t;
            const int64_t xa = da0 - i, xb = db0 - i;
            wA[t] = (i >= 0 && xa >= 0) ? XA[xa] : 0u;
            wB[t] = (i >= 0 && xb >= 0) ? XB[xb] : 0u;
        }
    } else {
        const int lane = tid;
        for (int j = lane; j < H; j += 32) {
            hAB[j] = da0 - j >= 0 ? XA[da0 - j] : 0u;
            hAB[GCD_HMAX + j] = db0 - j >= 0 ? XB[db0 - j] : 0u;
        }
        __syncwarp();
        // offsets (from the round's tops) of the leading coefficients and exact head lengths; the
        // degrees are below 2^30, so offsets and the test deg a >= deg b <=> ua - ub <= da0 - db0 fit
        // 32-bit integers
        const int Da = (int)da0, Db = (int)db0, D0 = Da - Db;
        int ua = 0, ub = 0, va = H, vb = H;
        uint32_t la = gcd_strip(hAB, ua, min(va, Da + 1), lane);
        uint32_t lb = gcd_strip(hAB + GCD_HMAX, ub, min(vb, Db + 1), lane);
        int k = 0, kind = -1;
        int64_t dg = -1;
        for (int guard = 0; guard < GCD_SMAX + 2; ++guard) {
            const bool a_zero = ua > Da, b_zero = ub > Db;
            if ((!a_zero && ua >= va) || (!b_zero && ub >= vb)) break;   // head exhausted: next round
            if (a_zero || b_zero) {
                kind = a_zero ? (b_zero ? GCD_IS_ZERO : GCD_IS_B) : GCD_IS_A;
                dg = a_zero ? (b_zero ? -1 : Db - ub) : Da - ua;
                break;
            }
            if (ua == Da || ub == Db) { kind = GCD_IS_ONE; dg = 0; break; }   // a nonzero constant
            if (k == s) break;
            // One step in one code path: the reduced polynomial r (a when deg a >= deg b) loses its
            // leading term to lc(d) r - lc(r) x^(deg r - deg d) d, d the other one; r[ur+j] pairs with
            // d[ud+j].  Entries past what the remaining steps can reach (plus GCD_HEXTRA) are left
            // stale and count as unknown: a round whose degrees drop that far ends early instead.
            const bool redA = ua - ub <= D0;
            const int offr = redA ? 0 : GCD_HMAX, offd = GCD_HMAX - offr;
            const int ur = redA ? ua : ub, ud = redA ? ub : ua;
            const int vr = redA ? va : vb, vd = redA ? vb : va;
            const int Dr = redA ? Da : Db;
            const uint32_t c1 = redA ? lb : la, c2n = p - (redA ? la : lb);
            const int sh = ud - ur;
            const int vr_new = min(min(vr, ur + vd - ud), ur + (s - k) + GCD_HEXTRA);
            // the next 32 entries first: the new leading coefficient is the first nonzero one
            const int i0h = ur + 1 + lane;
            // (entries below vr_new of r and below vr_new + sh of d: within the heads)
            const bool hok = PM_CHK(vr_new <= GCD_HMAX && vr_new + sh <= GCD_HMAX);
            const bool live = hok && i0h < vr_new;
            uint32_t v = gcd_comb<MONT>(c1, hAB[offr + (live ? i0h : 0)], c2n, hAB[offd + (live ? i0h + sh : 0)], md);
            v = live ? v : 0u;
            if (live) hAB[offr + i0h] = v;
            const unsigned msk = __ballot_sync(0xffffffffu, v != 0u);
            const int f = __ffs(msk) - 1;
            uint32_t lnew = __shfl_sync(0xffffffffu, v, f < 0 ? 0 : f);
#pragma unroll 4
            for (int i = i0h + 32; hok && i < vr_new; i += 32)
                hAB[offr + i] = gcd_comb<MONT>(c1, hAB[offr + i], c2n, hAB[offd + i + sh], md);
            if (lane == 0) {
                rc1[k] = c1;
                rc2[k] = c2n;
                rsig[k] = (ub - ua) * 2 + (redA ? 0 : 1);
            }
            int ur_new = ur + 1 + f;
            if (!msk) {   // 32 zeros: strip on from the entries the loop above wrote
                ur_new = min(ur + 33, min(vr_new, Dr + 1));
                __syncwarp();
                lnew = gcd_strip(hAB + offr, ur_new, min(vr_new, Dr + 1), lane);
            }
            if (redA) {
                ua = ur_new;
                va = vr_new;
                la = lnew;
            } else {
                ub = ur_new;
                vb = vr_new;
                lb = lnew;
            }
            ++k;
            __syncwarp();
        }
        if (lane == 0) {
            r_k = k;
            r_ua = ua;
            r_ub = ub;
            r_kind = kind;
            r_dg = dg;
        }
    }
    __syncthreads();

    const int K = r_k;
    const int ua = r_ua, ub = r_ub;
    const int Hh = min(max(ua, ub), H);
    const int lo = H - Hh, hi = H + GCD_T + Hh;

    // own window words in registers; shared copies are refreshed when the other polynomial needs them
    uint32_t ra[GCD_J], rb[GCD_J];
#pragma unroll
    for (int j = 0; j < GCD_J; ++j) {
        const int t = lo + tid + j * GCD_THREADS;
        ra[j] = t < hi ? wA[t] : 0u;
        rb[j] = t < hi ? wB[t] : 0u;
    }
    const int nj = (hi - lo + GCD_THREADS - 1) / GCD_THREADS;   // slots in use (block-uniform)
    int prev = -1;
    int code = K > 0 ? rsig[0] : 0;
    uint32_t c1 = K > 0 ? rc1[0] : 0u, c2n = K > 0 ? rc2[0] : 0u;
    for (int k = 0; k < K; ++k) {
        const int typ = code & 1;
        const int sig = code >> 1;   // arithmetic shift: floor, exact for even code - typ
        const uint32_t m1 = c1, m2 = c2n;
        if (k + 1 < K) {             // the next step's record, ahead of its use
            code = rsig[k + 1];
            c1 = rc1[k + 1];
            c2n = rc2[k + 1];
        }
        if (typ != prev) {
            if (prev == 0) {
#pragma unroll
                for (int j = 0; j < GCD_J; ++j) {
                    const int t = lo + tid + j * GCD_THREADS;
                    if (j < nj && t < hi) wA[t] = ra[j];
                }
            } else if (prev == 1) {
#pragma unroll
                for (int j = 0; j < GCD_J; ++j) {
                    const int t = lo + tid + j * GCD_THREADS;
                    if (j < nj && t < hi) wB[t] = rb[j];
                }
            }
            __syncthreads();
            prev = typ;
        }
        if (typ == 0) {
#pragma unroll
            for (int j = 0; j < GCD_J; ++j) {
                if (j < nj) {
                    const int t = lo + tid + j * GCD_THREADS;
                    const int tb = t + sig;
                    const uint32_t y = (tb >= 0 && tb < Wn) ? wB[tb] : 0u;
                    if (t < hi) ra[j] = gcd_comb<MONT>(m1, ra[j], m2, y, md);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < GCD_J; ++j) {
                if (j < nj) {
                    const int t = lo + tid + j * GCD_THREADS;
                    const int ta = t - sig;
                    const uint32_t y = (ta >= 0 && ta < Wn) ? wA[ta] : 0u;
                    if (t < hi) rb[j] = gcd_comb<MONT>(m1, rb[j], m2, y, md);
                }
            }
        }
    }
    // this block's T positions
#pragma unroll
    for (int j = 0; j < GCD_J; ++j) {
        const int t = lo + tid + j * GCD_THREADS;
        if (t >= H && t < H + GCD_T) {
            const int64_t i = i0 - H + t;
            const int64_t xa = da0 - i, xb = db0 - i;
            if (xa >= 0) YA[xa] = ra[j];
            if (xb >= 0) YB[xb] = rb[j];
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        GcdState s1 = s0;
        s1.steps_lo = s0.steps_lo + K;
        s1.rounds = s0.rounds + 1;
        if (r_kind >= 0) {
            s1.done = 1;
            s1.kind = r_kind;
            s1.dg = r_dg;
            s1.buf = ybuf;
        } else {
            s1.da = da0 - ua;
            s1.db = db0 - ub;
        }
        *sout = s1;
    }
}

// The monic gcd into g[0 .. glen-1] (zeros above its degree).
__global__ void gcd_final_kernel(const uint32_t* __restrict__ A0, const uint32_t* __restrict__ B0,
                                 const uint32_t* __restrict__ A1, const uint32_t* __restrict__ B1,
                                 const GcdState* __restrict__ st, uint32_t* __restrict__ g, int64_t glen, uint32_t p,
                                 uint64_t mu, int* status) {
    pdl_wait();  // the last round's arrays and state
    const GcdState s = *st;
    __shared__ uint32_t inv_s;
    const uint32_t* src = nullptr;
    if (s.kind == GCD_IS_A) src = s.buf ? A1 : A0;
    if (s.kind == GCD_IS_B) src = s.buf ? B1 : B0;
    if (threadIdx.x == 0) {
        uint32_t w = 0;
        if (src) {
            // lc^-1 mod p by the extended Euclidean algorithm
            int64_t r0 = p, r1 = src[s.dg], t0 = 0, t1 = 1;
            while (r1 != 0) {
                const int64_t qt = r0 / r1;
                int64_t tmp = r0 - qt * r1;
                r0 = r1;
                r1 = tmp;
                tmp = t0 - qt * t1;
                t0 = t1;
                t1 = tmp;
            }
            if (r0 == 1) w = (uint32_t)(t0 < 0 ? t0 + p : t0);
            else if (blockIdx.x == 0) atomicCAS(status, 0, (int)PM_ERR_INVALID_ARG);
        }
        inv_s = w;
    }
    __syncthreads();
    const uint32_t w = inv_s;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < glen; x += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = 0;
        if (src && x <= s.dg) v = barrett((uint64_t)src[x] * w, p, mu);
        else if (s.kind == GCD_IS_ONE && x == 0) v = 1;
        g[x] = v;
    }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

pm_status launch_gcd(const uint32_t* a, int64_t na, const uint32_t* b, int64_t nb, uint32_t* g, int64_t* deg_g,
                     uint32_t p, int s, cudaStream_t st, DeviceWorkspace* ws) {
    if (s < 1 || s > GCD_SMAX) return PM_ERR_INVALID_ARG;
    StreamScratch* sc = nullptr;
    pm_status rc = stream_scratch(ws, st, &sc);
    if (rc != PM_OK) return rc;
    const size_t wa = align256(sizeof(uint32_t) * (size_t)na), wb = align256(sizeof(uint32_t) * (size_t)nb);
    rc = ensure_scratch(&sc->gcd, &sc->gcd_bytes, 256 + 2 * (wa + wb), st, false);
    if (rc != PM_OK) return rc;
    char* base = reinterpret_cast<char*>(sc->gcd);
    GcdState* state = reinterpret_cast<GcdState*>(base);
    uint32_t* A[2] = {reinterpret_cast<uint32_t*>(base + 256), reinterpret_cast<uint32_t*>(base + 256 + wa)};
    uint32_t* B[2] = {reinterpret_cast<uint32_t*>(base + 256 + 2 * wa),
                      reinterpret_cast<uint32_t*>(base + 256 + 2 * wa + wb)};
    const uint64_t mu = (uint64_t)(((unsigned __int128)1 << 64) / p);
    GcdMod md{p, 0u, mu};
    if (p & 1u) {
        uint32_t inv = p;                       // Newton: each step doubles the correct low bits
        for (int i = 0; i < 5; ++i) inv *= 2u - p * inv;
        md.pinv = 0u - inv;
    }
    const int H = s + GCD_HEXTRA;
    const int64_t nmax = std::max(na, nb);
    uint64_t launches = 0;

    const int init_blocks = (int)std::min<int64_t>((nmax + 255) / 256, 4 * (int64_t)ws->num_sms);
    cudaError_t eb = chk_bind(ws);
    if (eb != cudaSuccess) return cuda_fail(eb);
    gcd_init_kernel<<<init_blocks, 256, 0, st>>>(a, na, b, nb, A[0], B[0], p, state);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    ++launches;

    int64_t da = na - 1, db = nb - 1, r = 0;
    const int64_t round_cap = na + nb + 4;   // every round lowers da + db by at least one
    GcdState host{};
    for (;;) {
        // enough rounds for da + db + 2 steps at s per round, plus one
        const int64_t batch = std::min<int64_t>((da + db + 2 + s - 1) / s + 1, round_cap - r);
        if (batch <= 0) return PM_ERR_INTERNAL;
        const unsigned blocks = (unsigned)std::max<int64_t>(1, (std::max(da, db) + GCD_T) / GCD_T);
        for (int64_t i = 0; i < batch; ++i, ++r) {
            const int x = (int)(r & 1), y = x ^ 1;
            e = launch_dep((p & 1u) ? gcd_round_kernel<true> : gcd_round_kernel<false>, dim3(blocks),
                           dim3(GCD_THREADS), 0, st, (const uint32_t*)A[x], (const uint32_t*)B[x], A[y], B[y],
                           (const GcdState*)(state + x), state + y, s, H, y, md);
            if (e != cudaSuccess) return cuda_fail(e);
            ++launches;
        }
        e = cudaMemcpyAsync(&host, state + (r & 1), sizeof(GcdState), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e);
        if (host.done) break;
        da = host.da;
        db = host.db;
    }
    const int final_blocks = (int)std::min<int64_t>((nmax + 255) / 256, 4 * (int64_t)ws->num_sms);
    e = launch_dep(gcd_final_kernel, dim3(std::max(1, final_blocks)), dim3(256), 0, st, (const uint32_t*)A[0],
                   (const uint32_t*)B[0], (const uint32_t*)A[1], (const uint32_t*)B[1],
                   (const GcdState*)(state + (r & 1)), g, nmax, p, mu, ws->status);
    if (e != cudaSuccess) return cuda_fail(e);
    ++launches;
    count_launches(launches);
    *deg_g = host.dg;
    return PM_OK;
}

}  // namespace pm
