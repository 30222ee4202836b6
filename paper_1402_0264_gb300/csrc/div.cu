// Euclidean division over Z/pZ (Section 3, "Polynomial division"): for a
// with n terms and b with m terms (n >= m >= 1, b's leading coefficient
// invertible mod p), the unique q (n-m+1 terms) and r (m-1 terms) with
// a = q b + r and deg r < deg b.
//
// Paper -> this file.  Algorithm 3 (OptimizePlainDivisionGPU) calls the
// kernel of Algorithm 4 (OptDivKer) once per s division steps, from the top
// coefficient down; each thread-block carries the s leading coefficients of
// the current remainder (its "s-head") through the s steps and updates its
// own stretch of the remainder below the head, redundantly with the other
// blocks for the head.  Here each launch of div_round_kernel is one such
// call, with the same split of the work:
//   head: one warp runs the round's division steps on the s-head (step k:
//         q_k = head[k] lc(b)^-1, then head[t] -= q_k b[d_b - (t - k)] for
//         t > k), 32 steps at a time with the group's entries in registers and
//         the later entries updated once per group, and keeps the s quotient
//         coefficients;
//   body: every other thread then applies all s steps to its positions at
//         once, r[x] -= sum_k q_k b[x - (i - k) + d_b], as a short convolution
//         summed lazily in 64 bits and reduced once per 8 terms (the same
//         final values as the paper's step-by-step updates: the updates are
//         linear and commute).
// Algorithm 1-2 (the naive division) is s = 1.  The s steps of a round and
// the rounds themselves are sequential (the span grows with n - m + 1, as in
// the paper's S_s = 3 (n - m + 1)); the parallelism is over the remainder's
// positions.
#include "common.cuh"

namespace pm {

#ifndef PM_DIV_THREADS
#define PM_DIV_THREADS 128   // measured: 128-thread blocks, one body position per thread
#endif
#ifndef PM_DIV_E
#define PM_DIV_E 1
#endif
constexpr int DIV_THREADS = PM_DIV_THREADS;
constexpr int DIV_E = PM_DIV_E;                  // remainder positions per thread in the body
constexpr int DIV_BODY = DIV_THREADS * DIV_E;    // positions below the head per block
constexpr int DIV_SMAX = 256;                    // largest s

__device__ __forceinline__ uint32_t div_sub(uint32_t x, uint32_t y, uint32_t p) {
    return x >= y ? x - y : x + (p - y);
}

// x w mod p for a constant w with Shoup's precomputed wq = floor(w 2^32 / p)
// (V. Shoup, NTL; D. Harvey, J. Symb. Comp. 2014): the estimate
// q = hi32(x wq) leaves x w - q p in [0, 2p).
__device__ __forceinline__ uint32_t div_mul_const(uint32_t x, uint32_t w, uint32_t wq, uint32_t p) {
    const uint32_t q = __umulhi(x, wq);
    const uint32_t r = x * w - q * p;
    return r >= p ? r - p : r;
}

// Working copy of a; lc(b)^-1 mod p by the extended Euclidean algorithm into
// inv[0] and its Shoup quotient into inv[1] (inv[0] = 0: no inverse).
__global__ void div_setup_kernel(const uint32_t* __restrict__ a, int64_t n, const uint32_t* __restrict__ b,
                                 int64_t d_b, uint32_t p, uint32_t* __restrict__ work, uint32_t* __restrict__ inv,
                                 int* status) {
    pdl_trigger();  // the first round may be placed now; it waits for this kernel to end
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        work[x] = a[x];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t r0 = p, r1 = b[d_b] % p, t0 = 0, t1 = 1;
        while (r1 != 0) {
            const int64_t qt = r0 / r1;
            int64_t tmp = r0 - qt * r1;
            r0 = r1;
            r1 = tmp;
            tmp = t0 - qt * t1;
            t0 = t1;
            t1 = tmp;
        }
        if (r0 != 1) {
            inv[0] = inv[1] = 0;
            atomicCAS(status, 0, (int)PM_ERR_INVALID_ARG);
        } else {
            const uint32_t w = (uint32_t)(t0 < 0 ? t0 + p : t0);
            inv[0] = w;
            inv[1] = (uint32_t)(((uint64_t)w << 32) / p);
        }
    }
}

// One round: division steps for the coefficients i, i-1, ... (at most s of
// them, down to d_b) of the remainder `work`.  Block g's body is the DIV_BODY
// positions below the head from top = i - s - g DIV_BODY down.
__global__ void __launch_bounds__(DIV_THREADS) div_round_kernel(uint32_t* __restrict__ work,
                                                                const uint32_t* __restrict__ b,
                                                                uint32_t* __restrict__ q, int64_t i, int64_t d_b,
                                                                int s, const uint32_t* __restrict__ inv, uint32_t p,
                                                                uint64_t mu) {
    __shared__ uint32_t head[DIV_SMAX];          // coefficients i - t of the remainder
    __shared__ uint32_t bh[DIV_SMAX];            // b[d_b - t]
    __shared__ uint32_t bhq[DIV_SMAX];           // its Shoup quotients floor(bh 2^32 / p)
    __shared__ uint32_t sq[DIV_SMAX];            // the round's quotient coefficients
    __shared__ uint32_t sb[DIV_BODY + DIV_SMAX]; // b window of the body
    // (uniform: before any barrier) the round's steps and the body window fit the shared arrays
    if (!PM_CHK(s >= 1 && s <= DIV_SMAX && blockDim.x == DIV_THREADS)) return;
    const int tid = threadIdx.x;
    const int ks = (int)min((int64_t)s, i - d_b + 1);  // division steps of this round
    const int64_t top = i - s - (int64_t)blockIdx.x * DIV_BODY;
    // b index of position x at step k is x - i + k + d_b; over this block's positions
    // (x = top - u, u < DIV_BODY) and k < s it runs over bx0 .. bx0 + DIV_BODY + s - 2
    const int64_t bx0 = top - i + d_b - (DIV_BODY - 1);
    // b is an input no kernel of the call writes: its windows are read before the
    // previous round has ended
    for (int t = tid; t < s; t += DIV_THREADS) {
        const uint32_t bv = d_b - t >= 0 ? b[d_b - t] : 0u;
        bh[t] = bv;
        bhq[t] = (uint32_t)(((uint64_t)bv << 32) / p);
    }
    for (int v = tid; v < DIV_BODY + s - 1; v += DIV_THREADS) {
        const int64_t bi = bx0 + v;
        sb[v] = (bi >= 0 && bi <= d_b) ? b[bi] : 0u;
    }
    pdl_wait();  // the previous round's remainder (or the setup's copy and inverse)
    pdl_trigger();
    const uint32_t w = inv[0], wq = inv[1];
    if (w == 0) return;  // b's leading coefficient has no inverse (status set by the setup)
    for (int t = tid; t < s; t += DIV_THREADS) head[t] = i - t >= 0 ? work[i - t] : 0u;
    __syncthreads();
    if (tid < 32) {  // the head: one warp, the steps in order
        // Steps in groups of 32: lane j holds head entry k0 + j of the group in a
        // register, so a step costs one shuffle and one product per lane on the
        // sequential path; the group's 32 quotient terms then update the entries
        // beyond the group at once.
        for (int k0 = 0; k0 < ks; k0 += 32) {
            const int kend = min(k0 + 32, ks);
            const int t = k0 + tid;
            uint32_t h = t < s ? head[t] : 0u;
            for (int k = k0; k < kend; ++k) {
                // branch-free: every lane stores the same q_k, and the update is a select
                const uint32_t qk = div_mul_const(__shfl_sync(0xffffffffu, h, k - k0), w, wq, p);
                sq[k] = qk;
                const bool live = t > k && t < s;
                const int j = live ? t - k : 0;
                const uint32_t upd = div_sub(h, div_mul_const(qk, bh[j], bhq[j], p), p);
                h = live ? upd : h;
            }
            if (t < s) head[t] = h;
            __syncwarp();
            for (int u = k0 + 32 + tid; u < s; u += 32) {  // entries after the group's 32
                uint64_t acc = 0;  // at most 32 reduced products: below 2^35
                for (int k = k0; k < kend; ++k) acc += div_mul_const(sq[k], bh[u - k], bhq[u - k], p);
                head[u] = div_sub(head[u], barrett(acc, p, mu), p);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        for (int t = tid; t < ks; t += DIV_THREADS) q[i - t - d_b] = sq[t];
        // head coefficients below d_b (last round only) are part of the remainder
        for (int t = ks + tid; t < s; t += DIV_THREADS)
            if (i - t >= 0) work[i - t] = head[t];
    }
    // the body: all steps of the round at once
#pragma unroll
    for (int e = 0; e < DIV_E; ++e) {
        const int u = tid + e * DIV_THREADS;
        const int64_t x = top - u;
        if (x < 0) continue;
        const uint32_t* bw = sb + (DIV_BODY - 1 - u);  // bw[k] = b[x - i + k + d_b]
        uint32_t total = 0;
        for (int k0 = 0; k0 < ks; k0 += 8) {
            uint64_t acc = 0;  // at most 8 products below p^2 < 2^60
            const int k1 = min(k0 + 8, ks);
            for (int k = k0; k < k1; ++k) acc += (uint64_t)sq[k] * bw[k];
            total += barrett(acc, p, mu);
            total = total >= p ? total - p : total;
        }
        work[x] = div_sub(work[x], total, p);
    }
}

pm_status launch_divide(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* q, uint32_t* r,
                        uint32_t p, int s, cudaStream_t st, DeviceWorkspace* ws) {
    if (s < 1 || s > DIV_SMAX) return PM_ERR_INVALID_ARG;
    StreamScratch* sc = nullptr;
    pm_status rc = stream_scratch(ws, st, &sc);
    if (rc != PM_OK) return rc;
    rc = ensure_scratch(&sc->div, &sc->div_bytes, 256 + sizeof(uint32_t) * (size_t)n, st, false);
    if (rc != PM_OK) return rc;
    uint32_t* inv = reinterpret_cast<uint32_t*>(sc->div);
    uint32_t* work = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(sc->div) + 256);
    const int64_t d_b = m - 1;
    const int setup_blocks = (int)std::min<int64_t>((n + 255) / 256, 4 * (int64_t)ws->num_sms);
    cudaError_t eb = chk_bind(ws);
    if (eb != cudaSuccess) return cuda_fail(eb);
    div_setup_kernel<<<setup_blocks, 256, 0, st>>>(a, n, b, d_b, p, work, inv, ws->status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    const uint64_t mu = (uint64_t)(((unsigned __int128)1 << 64) / p);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, (d_b + DIV_BODY - 1) / DIV_BODY);
    uint64_t launches = 1;
    for (int64_t i = n - 1; i >= d_b; i -= s, ++launches) {
        e = launch_dep(div_round_kernel, dim3(blocks), dim3(DIV_THREADS), 0, st, work, b, q, i, d_b, s,
                       (const uint32_t*)inv, p, mu);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (d_b > 0) {
        e = cudaMemcpyAsync(r, work, sizeof(uint32_t) * (size_t)d_b, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    count_launches(launches);
    return PM_OK;
}

}  // namespace pm
