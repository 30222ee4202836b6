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
// keeps it congruent mod p.  One application leaves at most
// (2^32-1)(c+1) with c = 2^32 mod p, two leave at most 2^32-1+c^2; the host
// picks one or two applications and the largest fold_every such that
// bound + fold_every * KB * (p-1)^2 < 2^64 (KB products per accumulator per
// sub-step), whichever costs fewer instructions per product.  The final value is reduced with Barrett's method
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
    int fold_twice;     // 1: a fold applies the map twice, 0: once
};

#ifndef PM_MACFORM
#define PM_MACFORM 0  // 0: C++ product + add, 1: mad.wide.u32, 2: mad.lo.cc/madc.hi pair
#endif
// acc + x*y with a 32x32->64 product
__device__ __forceinline__ uint64_t mad_wide(uint32_t x, uint32_t y, uint64_t acc) {
#if PM_MACFORM == 1
    uint64_t r;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(x), "r"(y), "l"(acc));
    return r;
#elif PM_MACFORM == 2
    uint32_t lo = (uint32_t)acc, hi = (uint32_t)(acc >> 32);
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;"
        : "+r"(lo), "+r"(hi) : "r"(x), "r"(y));
    return ((uint64_t)hi << 32) | lo;
#else
    return acc + (uint64_t)x * (uint64_t)y;
#endif
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
// The checked build (compiled with -DPOLYMUL_CHECKED into a library of its
// own; compute-sanitizer is not available to every user of this code).
// PM_CHK(cond) guards a global or shared-memory access: when cond fails it
// records PM_ERR_INTERNAL in the device status word and returns false, so the
// caller skips the access instead of faulting; in the normal build it is the
// constant true and costs nothing.  Each translation unit keeps the status
// word's address in a constant of its own, bound by chk_bind before its
// launches.
// ---------------------------------------------------------------------------
#ifdef POLYMUL_CHECKED
static __constant__ int* g_chk_status;
__device__ __forceinline__ bool pm_chk(bool ok) {
    if (!ok && g_chk_status) atomicCAS(g_chk_status, 0, (int)PM_ERR_INTERNAL);
    return ok;
}
#define PM_CHK(cond) pm_chk(cond)
#else
#define PM_CHK(cond) true
#endif

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
ModParams host_mod_params(uint32_t p, int kb);

// Scratch owned by the library for one (device, stream): calls on one stream
// are ordered, so they can share it; calls on different streams never do.
struct StreamScratch {
    void* sk = nullptr;            // partial-sum slots and counters of the plain kernels
    size_t sk_bytes = 0;
    void* plan = nullptr;          // position prefix of polymul_batched
    size_t plan_bytes = 0;
    void* tc = nullptr;            // tensor-core path scratch
    size_t tc_bytes = 0;
    void* ntt = nullptr;           // transform buffers
    size_t ntt_bytes = 0;
    void* div = nullptr;           // division: working copy of the dividend, inverse of lc(b)
    size_t div_bytes = 0;
    void* gcd = nullptr;           // gcd: round states and two copies of both polynomials
    size_t gcd_bytes = 0;
};

// Per-device state owned by the library.
struct DeviceWorkspace {
    int device = -1;
    int num_sms = 0;
    int cc_major = 0, cc_minor = 0;
    int* status = nullptr;          // device status word (pm_status), zero = PM_OK
    void* twiddles = nullptr;       // transform twiddle tables (read-only, shared by streams)
    size_t twiddle_bytes = 0;
    uint32_t tw_p = 0, tw_g = 0;    // modulus/generator the tables were built for
    int tw_logn = -1;
    void* streams = nullptr;        // map cudaStream_t -> StreamScratch* (api.cu)
};

// Returns the workspace of the current device, creating it on first use.
// Never allocates while `stream` is capturing (returns null then).
DeviceWorkspace* workspace(void* stream, pm_status* err);
// The scratch of (ws's device, stream), created on first use.
pm_status stream_scratch(DeviceWorkspace* ws, cudaStream_t st, StreamScratch** out);
// Grows *buf to at least `bytes` (cudaMalloc; refused during capture); when it
// allocates and `zero` is set, clears the new buffer on `st`.
pm_status ensure_scratch(void** buf, size_t* have, size_t bytes, cudaStream_t st, bool zero);

pm_status cuda_fail(cudaError_t e);

// Checked build: points this translation unit's status constant at the device's
// status word (once per device); a no-op otherwise.
static inline cudaError_t chk_bind(DeviceWorkspace* ws) {
#ifdef POLYMUL_CHECKED
    static int bound[64] = {};
    if (ws->device >= 0 && ws->device < 64 && !bound[ws->device]) {
        cudaError_t e = cudaMemcpyToSymbol(g_chk_status, &ws->status, sizeof(int*));
        if (e != cudaSuccess) return e;
        bound[ws->device] = 1;
    }
#else
    (void)ws;
#endif
    return cudaSuccess;
}

// cudaMalloc, unless a test has asked for the next allocations to fail
// (polymul_debug_set(PM_DEBUG_FAIL_ALLOC, k)).
cudaError_t dev_alloc(void** ptr, size_t bytes);
// Polls before a wait of the tensor-core kernel is declared lost; 0 = built-in
// limit (polymul_debug_set(PM_DEBUG_TC_WAIT_LIMIT, k)).
int64_t tc_wait_limit();
void release_ntt_tables();
void release_host_io();
void count_launches(uint64_t k);
bool is_capturing(void* stream);

// Programmatic dependent launch between the kernels of one call.  A kernel
// launched by launch_dep may be scheduled while the kernel before it on the
// stream still runs; pdl_wait, before its first access to global memory,
// blocks until that kernel has completed and its writes are visible, so only
// the launch, the placement of its blocks and their set-up in shared and
// tensor memory overlap the previous kernel (no global memory access does).  pdl_trigger, at the start of the previous kernel, lets that
// placement begin once every block of it has started.  The first kernel of a
// call is launched the ordinary way, after everything queued before it.
#ifndef PM_PDL
#define PM_PDL 1
#endif
__device__ __forceinline__ void pdl_wait() {
#if PM_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_trigger() {
#if PM_PDL
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
#if PM_PDL
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
#else
    kernel<<<grid, block, smem, st>>>(args...);
    return cudaGetLastError();
#endif
}

// Pairs of a batch given to the plain launcher with max_short = PM_ALL_PAIRS are all computed; with a
// finite max_short only those whose shorter operand has fewer than max_short terms (the others are
// left to the tensor-core launcher, min_short = max_short).
constexpr int64_t PM_ALL_PAIRS = INT64_MAX;
// PM_AUTO's split between the forms: the shorter operand's terms from which a pair goes to the
// tensor cores (4096 pairs of degrees log-uniform in [16, 2048], ms: split 128 0.162, 256 0.168,
// 512 0.167, 1024 0.192; the plain form alone 0.184, the tensor form alone 0.191)
#ifndef PM_AUTO_SPLIT
#define PM_AUTO_SPLIT 128
#endif

// Kernel launchers (one translation unit each).
pm_status launch_plain(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* c,
                       uint32_t p, int s, cudaStream_t st, DeviceWorkspace* ws);
// q_min: the smallest unit (positions) of the warp-level schedule; 0 = the default
pm_status launch_batched_plain(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                               const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                               const int64_t* c_off, uint32_t p, int s, int64_t max_deg, int64_t q_min,
                               int64_t max_short,
                               cudaStream_t st, DeviceWorkspace* ws);
pm_status launch_ntt(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* c,
                     uint32_t p, uint32_t g, cudaStream_t st, DeviceWorkspace* ws);
pm_status launch_batched_tensor(int64_t batch, const uint32_t* a_data, const int64_t* a_off,
                                const uint32_t* b_data, const int64_t* b_off, uint32_t* c_data,
                                const int64_t* c_off, uint32_t p, int64_t max_deg, int64_t min_short,
                                cudaStream_t st, DeviceWorkspace* ws);
pm_status launch_mma_probe(int kind, int64_t iters, double* flops_per_clk_sm, int* exact, cudaStream_t st,
                           DeviceWorkspace* ws);
pm_status launch_plain_ell(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* c, uint32_t p,
                           int s, int ell, cudaStream_t st, DeviceWorkspace* ws);
pm_status launch_divide(const uint32_t* a, int64_t n, const uint32_t* b, int64_t m, uint32_t* q, uint32_t* r,
                        uint32_t p, int s, cudaStream_t st, DeviceWorkspace* ws);
pm_status launch_gcd(const uint32_t* a, int64_t na, const uint32_t* b, int64_t nb, uint32_t* g, int64_t* deg_g,
                     uint32_t p, int s, cudaStream_t st, DeviceWorkspace* ws);

}  // namespace pm
