// Shared device helpers of libpolymul: modular reduction for the lazy
// 64-bit accumulation, launch bookkeeping and the per-device workspace.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "polymul.h"

namespace pm {

// ---------------------------------------------------------------------------
// Modular parameters of one call, computed on the host (see host_mod_params).
//
// Accumulation scheme (the paper counts one field operation per word,
// Section 3; it does not say how sums are formed): products a*b < p^2 are
// summed unreduced in 64 bits.  Every `fold_every` sub-steps the sum is
// folded twice with x -> (x mod 2^32) + floor(x / 2^32) * (2^32 mod p), which
// keeps it congruent mod p and brings it below fold_bound, so that
// fold_bound + fold_every * KB * (p-1)^2 < 2^64 always holds (KB products per
// accumulator per sub-step).  The final value is reduced with Barrett's method
// (P. Barrett, "Implementing the RSA public key encryption algorithm on a
// standard digital signal processor", CRYPTO 1986): q = floor(x * mu / 2^64)
// with mu = floor(2^64 / p) underestimates floor(x / p) by at most one, so
// r = x - q p lies in [0, 2p) and one conditional subtraction finishes it.
// ---------------------------------------------------------------------------
struct ModParams {
    uint32_t p;
    uint32_t c32;       // 2^32 mod p
    uint64_t mu;        // floor(2^64 / p)
    int fold_every;     // sub-steps (of KB products) between two folds
    int pad_;
};

__device__ __forceinline__ uint64_t mad_wide(uint32_t x, uint32_t y, uint64_t acc) {
    uint64_t r;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(x), "r"(y), "l"(acc));
    return r;
}

__device__ __forceinline__ uint64_t fold_once(uint64_t x, uint32_t c32) {
    return mad_wide((uint32_t)(x >> 32), c32, x & 0xffffffffull);
}

__device__ __forceinline__ uint64_t fold2(uint64_t x, uint32_t c32) {
    return fold_once(fold_once(x, c32), c32);
}

__device__ __forceinline__ uint32_t barrett(uint64_t x, uint32_t p, uint64_t mu) {
    uint64_t q = __umul64hi(x, mu);
    uint64_t r = x - q * (uint64_t)p;
    return (uint32_t)(r >= p ? r - p : r);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
ModParams host_mod_params(uint32_t p, int kb);

// Per-device workspace owned by the library.
struct DeviceWorkspace {
    int device = -1;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    int* status = nullptr;          // device status word (pm_status), zero = PM_OK
    void* batch_ws = nullptr;       // work list of polymul_batched
    size_t batch_ws_bytes = 0;
    void* ntt_ws = nullptr;         // twiddle tables and transform scratch
    size_t ntt_ws_bytes = 0;
    uint32_t ntt_p = 0, ntt_g = 0;  // modulus/generator the tables were built for
    int ntt_logN = -1;
};

// Returns the workspace of the current device, creating it on first use.
// Never allocates while `stream` is capturing (returns null then).
DeviceWorkspace* workspace(void* stream, pm_status* err);
// Grows *buf to at least `bytes` (cudaMalloc; refused during capture).
pm_status ensure_buffer(void** buf, size_t* have, size_t bytes, void* stream);

pm_status cuda_fail(cudaError_t e);
void count_launches(uint64_t k);
bool is_capturing(void* stream);

// Kernel launchers (one translation unit each).
pm_status launch_plain(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* c,
                       uint32_t p, int s, cudaStream_t st, const DeviceWorkspace* ws);
pm_status launch_batched_plain(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                               const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                               const int64_t* c_off, uint32_t p, int s, int64_t max_deg,
                               cudaStream_t st, DeviceWorkspace* ws);
pm_status launch_ntt(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* c,
                     uint32_t p, uint32_t g, cudaStream_t st, DeviceWorkspace* ws);
pm_status launch_batched_tensor(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                                const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                                const int64_t* c_off, uint32_t p, int64_t max_deg,
                                cudaStream_t st, DeviceWorkspace* ws);

}  // namespace pm
