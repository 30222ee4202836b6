/*
 * polymul.h - C ABI of libpolymul.so: dense univariate polynomial
 * multiplication modulo a word-size prime on one NVIDIA GB300 (sm_103a).
 *
 * The operation (Haque, Moreno Maza, Xie, "A Many-core Machine Model for
 * Designing Algorithms with Minimum Parallelism Overheads", Section 5, with
 * the field and term conventions of Section 3): for a, b in K[X], K = Z/pZ,
 * with n = deg a + 1 and m = deg b + 1 terms ("null or not"),
 *
 *     c[k] = sum_{i+j=k, 0<=i<n, 0<=j<m} a[i] * b[j]  mod p,   0 <= k < n+m-1.
 *
 * Conventions shared by every entry point
 *   - Coefficients are uint32 in little-endian degree order (index = degree).
 *     Inputs must be < p; outputs are canonical residues in [0, p).
 *   - The output always has n+m-1 words; leading zeros are kept.
 *   - Array arguments are DEVICE pointers (cudaMalloc'd or torch tensors),
 *     owned by the caller.  The output must not overlap either input.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered and asynchronous: the return value
 *     covers argument validation and the kernel launch only.  Errors raised
 *     inside a kernel (a bounded wait that ran out) are recorded in a
 *     per-device status word read by polymul_sync_status().
 *   - The library owns a small per-device workspace (work lists, twiddle
 *     tables, status word), grown on demand with cudaMalloc and freed by
 *     polymul_release().  A call that would have to grow it while `stream`
 *     is being captured into a CUDA graph returns PM_ERR_UNSUPPORTED: make
 *     one uncaptured call of the same shape first.  A buffer replaced by a
 *     larger one is kept (not freed) until polymul_release(), so a graph
 *     captured before the growth stays valid.  Destroy every graph that holds
 *     library calls before polymul_release(), and do not replay such a graph
 *     while direct calls run on its capture stream's scratch (the same stream
 *     the calls were captured on) from another stream.
 *   - Thread safety: calls from several host threads are allowed; workspace
 *     growth is serialised by a lock.  Calls that share a device and run
 *     concurrently on different streams must not share output buffers.  A
 *     call's launches use its stream's scratch, so two host threads must not
 *     issue calls on the same stream at the same time (their launches could
 *     interleave); give each thread its own stream.
 */
#ifndef POLYMUL_H
#define POLYMUL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PM_OK = 0,
    PM_ERR_INVALID_ARG = 1,  /* null pointer, bad degree, bad s or mode, overlap, bad offsets */
    PM_ERR_RANGE = 2,        /* a size or modulus outside the supported range */
    PM_ERR_UNSUPPORTED = 3,  /* valid request this path cannot serve (e.g. no 2^k root of unity) */
    PM_ERR_NOMEM = 4,        /* workspace allocation failed */
    PM_ERR_CUDA = 5,         /* a CUDA runtime call failed; see polymul_last_cuda_error() */
    PM_ERR_TIMEOUT = 6,      /* a kernel's bounded wait ran out (reported by polymul_sync_status) */
    PM_ERR_INTERNAL = 7
} pm_status;

/* Modes of polymul_batched. */
#define PM_AUTO 0    /* each pair by its size: tensor cores for the larger, plain for the smaller */
#define PM_PLAIN 1   /* s-blocked CUDA-core product */
#define PM_TENSOR 2  /* bf16-limb Toeplitz product on the tcgen05 tensor cores */

/* Largest supported modulus (exclusive) and degree (inclusive). */
#define PM_MAX_P (1u << 30)
#define PM_MAX_DEG ((int64_t)(1 << 30) - 2)
/* Largest degree the tensor-core form takes (polymul_batched, PM_TENSOR). */
#define PM_TENSOR_MAX_DEG ((int64_t)(1 << 24) - 1)

/*
 * polymul_plain - one product by the s-blocked long multiplication
 * (Section 5, Algorithms 5-7: the multiplication phase forms s x s blocks of
 * partial products per thread, the addition phase sums them; here both
 * phases are fused in one kernel and the partial sums never leave the chip).
 *
 *   a, deg_a   device array of deg_a+1 coefficients (0 <= deg_a <= PM_MAX_DEG)
 *   b, deg_b   device array of deg_b+1 coefficients (0 <= deg_b <= PM_MAX_DEG)
 *   c          device array of deg_a+deg_b+1 words, written in full
 *   p          modulus, 2 <= p < PM_MAX_P (need not be prime)
 *   s          per-thread block parameter: 1, 2, 4, 8, 16, 32 or 64; 0 picks
 *              the tuned value for this size (polymul_tune_plain) or a default
 *   stream     cudaStream_t as void*
 * Returns PM_OK, PM_ERR_INVALID_ARG (pointers, degrees, s, c overlapping an
 * input), PM_ERR_RANGE (p), PM_ERR_UNSUPPORTED (scratch growth while the
 * stream captures), PM_ERR_NOMEM or PM_ERR_CUDA.
 */
pm_status polymul_plain(const uint32_t *a, int64_t deg_a, const uint32_t *b, int64_t deg_b,
                        uint32_t *c, uint32_t p, int s, void *stream);

/*
 * polymul_plain_ell - polymul_plain with a chosen number of threads per
 * block, the paper's l (Section 5: l threads per thread-block, each forming
 * s outputs; with s and U it fixes the model's N_s, L_s, C_s).  For the
 * study of the model's predictions over (s, l); the result is the same.
 *
 *   ell        128, 256 (polymul_plain's block) or 512
 *   s          1, 2, 4, 8, 16, 32 or 64 (no tuned default)
 *   other arguments as for polymul_plain.
 * At ell = 512 a thread may hold 128 registers, and s = 64 then keeps its
 * window of a in local memory (exact, but about 19x slower than ell = 256).
 * Returns PM_OK, PM_ERR_INVALID_ARG, PM_ERR_RANGE, PM_ERR_UNSUPPORTED,
 * PM_ERR_NOMEM or PM_ERR_CUDA.
 */
pm_status polymul_plain_ell(const uint32_t *a, int64_t deg_a, const uint32_t *b, int64_t deg_b,
                            uint32_t *c, uint32_t p, int s, int ell, void *stream);

/*
 * polymul_plain_noalloc - polymul_plain for callers that cannot allocate.
 * The paper has no counterpart: this is a deployment variant of the same
 * product.  Some callers cannot let a library call cudaMalloc: processes whose
 * caching allocator (PyTorch's, for one) has already reserved nearly all
 * device memory, so that a library's own cudaMalloc would fail; latency-bound
 * callers that cannot take the device-wide synchronisation that cudaMalloc and
 * cudaFree may imply; and hosts whose memory policy gives every allocation to
 * one owner.  This entry point allocates nothing: the kernel's scratch
 * (partial-sum slots and tile counters) lives in a 4 MiB static device array
 * that every GPU loading the library holds until the process exits.
 *
 *   Arguments, layout and result are those of polymul_plain.
 *   The first call on each device looks up the array's device address and
 *   clears its counters (synchronously, on the legacy default stream); make
 *   that first call before any stream capture (made while `stream` captures,
 *   it returns PM_ERR_UNSUPPORTED and does nothing).  Later calls only launch
 *   the kernel.
 *   All calls share the one array (its contents persist between calls; the
 *   kernel leaves its counters at zero), so calls whose kernels overlap on
 *   the GPU - on different streams, or from different host threads - race and
 *   give wrong results: serialise them.
 *   Returns PM_ERR_RANGE when the scratch a launch needs (2 slots of 32*s
 *   words per persistent CTA, plus the counters) would exceed the 4 MiB
 *   array; on GB300 every s fits.  Otherwise as polymul_plain.
 */
pm_status polymul_plain_noalloc(const uint32_t *a, int64_t deg_a, const uint32_t *b, int64_t deg_b,
                                uint32_t *c, uint32_t p, int s, void *stream);

/*
 * polymul_ntt - one product through number-theoretic transforms: forward
 * transforms of a and b zero-padded to N = 2^ceil(log2(n+m-1)), pointwise
 * product, inverse transform, scaling by N^-1 mod p.  Exact, so the result
 * equals polymul_plain's word for word.  (The paper has no transform path;
 * this is the large-degree path of the same product.)
 *
 *   p must be prime with N | p-1 and g a generator of (Z/pZ)^*; pass g = 0
 *   for p = 469762049 (7*2^26+1, generator 3).  N <= 2^24 (n+m-1 <= 2^24).
 *   Uses 8N bytes of library scratch per (device, stream) for N > 4096.
 * Returns PM_OK, PM_ERR_INVALID_ARG, PM_ERR_RANGE (N > 2^24),
 * PM_ERR_UNSUPPORTED (N does not divide p-1, no generator known, or g has
 * the wrong order), PM_ERR_NOMEM (tables, scratch) or PM_ERR_CUDA.
 */
pm_status polymul_ntt(const uint32_t *a, int64_t deg_a, const uint32_t *b, int64_t deg_b,
                      uint32_t *c, uint32_t p, uint32_t g, void *stream);

/*
 * polymul_batched - `batch` independent products, one stream-ordered sequence
 * of launches (planning kernels, then one persistent product kernel).
 *
 *   a_data, a_off  CSR: pair i's a is a_data[a_off[i] .. a_off[i+1]), at least one word
 *   b_data, b_off  likewise for b
 *   c_data, c_off  pair i's product goes to c_data[c_off[i] .. c_off[i+1]),
 *                  which must hold exactly n_i + m_i - 1 words
 *   The offset arrays (batch+1 int64 each) are DEVICE arrays, so the call can
 *   be captured into a CUDA graph; they are validated on the device and a bad
 *   layout sets PM_ERR_INVALID_ARG in the status word.
 *   p              2 <= p < PM_MAX_P (PM_TENSOR: also see below)
 *   mode           PM_PLAIN, PM_TENSOR or PM_AUTO
 *   s              as for polymul_plain (PM_PLAIN / PM_AUTO); ignored by PM_TENSOR
 *   max_deg        an upper bound on every degree in the batch (the host cannot
 *                  read the device offsets); PM_TENSOR needs max_deg <= PM_TENSOR_MAX_DEG
 * PM_PLAIN is the s-blocked product of Section 5 with the positions of the
 * whole batch shared out: when max_deg <= 4095 and s <= 32 each warp works on
 * its own units (a small pair, or a piece of a large one), claimed from a
 * counter; otherwise each persistent CTA takes an equal range of positions.
 * The warp-level form holds up to 64 MiB of scratch per (device, stream).
 * PM_TENSOR computes the same residues on the tensor cores (bf16 limbs, fp32
 * accumulation that stays exact below 2^24: pairs whose shorter operand has
 * more terms than one accumulation may sum, max_terms of polymul_tensor_limbs,
 * are accumulated in groups of at most that many terms and the groups'
 * residues added); it needs p < 2^29 and
 * max_deg <= PM_TENSOR_MAX_DEG, else returns PM_ERR_UNSUPPORTED.  PM_AUTO,
 * where the tensor cores apply, sends each pair by its size: pairs whose
 * shorter operand has at least 128 terms to the tensor cores and the others
 * to the warp-level plain form (both launched on `stream`, each skipping the
 * other's pairs), or, when max_deg > 4095 or the plain s is 64, the whole
 * batch to the tensor cores; where they do not apply, the plain form.
 * With s = 0 the plain form takes the tuned (s, Q) of the batch's size class
 * (polymul_tune_batched), else the tuned s of a single pair of degree max_deg
 * (polymul_tune_plain), else 8 from max_deg 1023 up, 4 from 63, else 2.
 * Returns PM_OK, PM_ERR_INVALID_ARG, PM_ERR_UNSUPPORTED, PM_ERR_NOMEM or PM_ERR_CUDA.
 */
pm_status polymul_batched(int64_t batch, const uint32_t *a_data, const int64_t *a_off,
                          const uint32_t *b_data, const int64_t *b_off,
                          uint32_t *c_data, const int64_t *c_off, uint32_t p,
                          int mode, int s, int64_t max_deg, void *stream);

/*
 * polymul_batched_host - polymul_batched from and to HOST buffers: the same
 * arguments, with a_data, a_off, b_data, b_off, c_data and c_off in host
 * memory (page-locked memory, cudaHostAlloc / cudaHostRegister, lets the
 * copies run asynchronously and overlap; pageable memory works, slower).  The
 * batch is cut into up to 4 chunks of consecutive pairs with about equal
 * multiply-adds; each chunk's words are copied to the device, multiplied by
 * polymul_batched (same mode, s and max_deg) and copied back, on three streams
 * of the library's own (per device), so that the copies of one chunk overlap
 * the products of the next.  Stream order: the copies start after the work
 * queued on `stream` before the call, and work queued on `stream` after it
 * runs once every product is back in c_data; the host buffers must stay
 * valid, and the inputs unchanged, until then.  The device buffers (two chunk
 * slots) are the library's, grown when a larger chunk needs it and freed by
 * polymul_release.  The offsets are checked on the host (the same layout rules
 * as polymul_batched; PM_ERR_INVALID_ARG), and c_data may not overlap a_data
 * or b_data.  Not capturable: returns PM_ERR_UNSUPPORTED while `stream`
 * captures.  (No counterpart in the paper: the end-to-end form of the batched
 * product.)
 * Returns PM_OK, PM_ERR_INVALID_ARG, PM_ERR_RANGE, PM_ERR_UNSUPPORTED,
 * PM_ERR_NOMEM or PM_ERR_CUDA; kernel-side errors go to the status word.
 */
pm_status polymul_batched_host(int64_t batch, const uint32_t *a_data, const int64_t *a_off,
                               const uint32_t *b_data, const int64_t *b_off, uint32_t *c_data,
                               const int64_t *c_off, uint32_t p, int mode, int s, int64_t max_deg,
                               void *stream);

/*
 * polymul_divide - Euclidean division over Z/pZ (Section 3, "Polynomial
 * division", Algorithms 3-4 with parameter s; s = 1 is the naive division of
 * Algorithms 1-2): the unique q and r with a = q b + r and deg r < deg b.
 *
 *   a, deg_a   device array of deg_a+1 coefficients, deg_b <= deg_a <= PM_MAX_DEG
 *   b, deg_b   device array of deg_b+1 coefficients; b[deg_b] must be invertible
 *              mod p (nonzero when p is prime)
 *   q          device array of deg_a-deg_b+1 words, written in full
 *   r          device array of deg_b words (the remainder's deg_b low terms,
 *              leading zeros kept); may be NULL when deg_b = 0
 *   p          2 <= p < PM_MAX_P (need not be prime)
 *   s          division steps per kernel launch, 1 <= s <= 256; 0 picks 128
 *   stream     cudaStream_t as void*
 * The steps run from the top coefficient down, s per launch (one launch per
 * s quotient terms, after one set-up launch), so the call is stream-ordered
 * and can be captured into a CUDA graph once its scratch (4 (deg_a + 1) + 256
 * bytes per (device, stream)) exists.  A leading coefficient of b without an
 * inverse sets PM_ERR_INVALID_ARG in the status word (polymul_sync_status);
 * q and r are then undefined.
 * Returns PM_OK, PM_ERR_INVALID_ARG (null pointer, degrees, s, overlapping
 * arrays), PM_ERR_RANGE (p), PM_ERR_NOMEM or PM_ERR_CUDA.
 */
pm_status polymul_divide(const uint32_t *a, int64_t deg_a, const uint32_t *b, int64_t deg_b,
                         uint32_t *q, uint32_t *r, uint32_t p, int s, void *stream);

/*
 * polymul_gcd - the monic greatest common divisor over Z/pZ (Section 6,
 * "The Euclidean algorithm for polynomials", Algorithms 10-11 with parameter
 * s; s = 1 is the naive gcd of Algorithms 8-9, one division step per launch).
 *
 *   a, deg_a   device array of deg_a+1 coefficients (0 <= deg_a <= PM_MAX_DEG);
 *              leading zeros allowed, words are taken mod p
 *   b, deg_b   the same for b; a = 0 or b = 0 is allowed
 *   g          device array of max(deg_a, deg_b)+1 words, written in full: the
 *              monic gcd in g[0 .. *deg_g], zeros above it (all zeros when
 *              a = b = 0)
 *   deg_g      host pointer: the degree of the gcd, -1 when a = b = 0
 *   p          prime, 2 <= p < PM_MAX_P (primality is not checked; a leading
 *              coefficient without an inverse sets PM_ERR_INVALID_ARG in the
 *              status word)
 *   s          division steps per launch, 1 <= s <= 256; 0 picks 64
 *   stream     cudaStream_t as void*
 * The number of division steps (at most deg_a + deg_b + 2) depends on the
 * data, so the call launches rounds of s steps in batches and reads a
 * 48-byte state back after each batch: it synchronises `stream` and cannot
 * be captured into a CUDA graph (PM_ERR_UNSUPPORTED while capturing).
 * Scratch: 8 (deg_a + deg_b + 2) bytes plus 1 KiB per (device, stream).
 * Returns PM_OK, PM_ERR_INVALID_ARG (null pointer, degrees, s, g overlapping
 * an input), PM_ERR_RANGE (p), PM_ERR_UNSUPPORTED, PM_ERR_NOMEM,
 * PM_ERR_INTERNAL or PM_ERR_CUDA.
 */
pm_status polymul_gcd(const uint32_t *a, int64_t deg_a, const uint32_t *b, int64_t deg_b, uint32_t *g,
                      int64_t *deg_g, uint32_t p, int s, void *stream);

/*
 * polymul_model_predict - the cost model of the s-blocked product
 * (Section 5 printed formulas; Theorem 1 and Corollary 1 of Section 2.4).
 * Host-only; no GPU needed.
 *
 *   n, m   numbers of terms of a and b;  s, ell  block parameter and threads per block
 *   U      cycles to move one word between global and local memory, in units of one
 *          local operation (the machine parameter of Section 2.1)
 *   P      number of streaming multiprocessors for Theorem 1
 *   out    9 doubles: W_s, S_s, O_s, N_s, L_s, C_s, K (MulKer blocks),
 *          T_thm = (N_s/P + L_s) C_s, T_cor = (N_s/K + L_s) C_s
 * Returns PM_OK or PM_ERR_INVALID_ARG (n, m, s, ell < 1, s > m, U or P <= 0, out NULL).
 */
pm_status polymul_model_predict(int64_t n, int64_t m, int s, int ell, double U, double P,
                                double *out);

/*
 * polymul_tune_plain - the autotuner of the block parameter s (the paper's
 * strategy, Section 2.4 and Section 5: the s that the measured time favours
 * among those the model allows).  For every s in {1,2,4,8,16,32,64} it
 * makes one warm-up call, then `reps` timed calls (CUDA events around each
 * one, after a write of twice the L2 size so that each call starts from HBM)
 * on the caller's buffers, and takes the median.  The chosen s is the
 * smallest one within 2% of the fastest median (near-ties go to the smaller
 * block); it is recorded in the tuners' cache (below) for this size class
 * (device model, log2 buckets of n and m, and p below or above 2^29) so that
 * later s = 0 calls use it.  The per-s medians
 * go to times_ms[7] (may be NULL; -1 where s exceeds both lengths) and the
 * choice to *best_s.  Allocates (and frees) the flush buffer; synchronises
 * `stream`.  reps >= 20 gives stable medians.
 * Returns what polymul_plain returns, PM_ERR_NOMEM or PM_ERR_CUDA.
 */
pm_status polymul_tune_plain(const uint32_t *a, int64_t deg_a, const uint32_t *b, int64_t deg_b,
                             uint32_t *c, uint32_t p, int reps, void *stream, int *best_s,
                             float *times_ms);

/* Returns the s that an s = 0 call of polymul_plain would use for these sizes. */
int polymul_plain_default_s(int64_t deg_a, int64_t deg_b, uint32_t p);

/*
 * polymul_tune_batched - the autotuner of the batched plain form (Section 5's
 * block parameter s, applied per size class of a batch).  Arguments as for
 * polymul_batched (the caller's buffers; c_data is overwritten).  For batches
 * with max_deg <= 4095 it times the warp-level schedule for s in {2, 4, 8, 16}
 * and unit sizes Q in {128, 256, 512, 1024, 2048} positions (the smallest
 * piece a pair is cut into; Q also sets the claim tiers); above that, the CTA
 * form for every s.  Each candidate: one warm-up call, then `reps` calls each
 * after a write of twice the L2 size, the median kept.  The choice is the
 * smallest s (then the smallest Q) within 2% of the fastest median; it is
 * recorded for this size class (device model, p below or above 2^29, log2 of
 * max_deg + 1 and of the batch size) and used by later calls of
 * polymul_batched with mode PM_PLAIN or PM_AUTO's plain path and s = 0 (an
 * explicit s keeps the tuned Q only if it equals the tuned s).  times_ms (may
 * be NULL) receives 35 medians, index 5 i + j for s = 2^i and Q = 128 * 2^j
 * (the CTA form: j = 1), -1 where not timed.  Allocates (and frees) the flush
 * buffer; synchronises `stream`.
 * Returns PM_OK, PM_ERR_INVALID_ARG (arguments, reps < 1, or the device
 * status word set after the runs: a bad layout), PM_ERR_UNSUPPORTED (the
 * stream captures), PM_ERR_NOMEM, PM_ERR_CUDA or PM_ERR_INTERNAL.
 */
pm_status polymul_tune_batched(int64_t batch, const uint32_t *a_data, const int64_t *a_off,
                               const uint32_t *b_data, const int64_t *b_off, uint32_t *c_data,
                               const int64_t *c_off, uint32_t p, int64_t max_deg, int reps, void *stream,
                               int *best_s, int64_t *best_q, float *times_ms);

/*
 * The tuners' cache.  Every choice polymul_tune_plain and polymul_tune_batched
 * make is kept in a process-wide table keyed by the device's name and SM
 * count, the form (PM_TUNE_PLAIN: one product, buckets floor(log2 n) and
 * floor(log2 m) of the longer and shorter operand; PM_TUNE_BATCHED: buckets
 * floor(log2(max_deg + 1)) and floor(log2 batch)) and whether p >= 2^29.
 * If the environment variable POLYMUL_TUNE_CACHE names a file when the table
 * is first used, that file is loaded (a missing or unreadable file is
 * ignored).  Host-only; no GPU needed.
 *
 *   polymul_tune_save    writes the table as JSON ({"version": 1, "entries":
 *                        [...]}, one object per choice) to `path` (through a
 *                        temporary file and a rename)
 *   polymul_tune_load    adds the entries of a file written by
 *                        polymul_tune_save (replacing equal keys); entries of
 *                        other devices are kept and used only on such devices
 *   polymul_tune_clear   empties the table (and skips the environment's file)
 *   polymul_tune_lookup  the choice stored for an explicit device name, SM
 *                        count, form, p and sizes (x, y = n, m or max_deg + 1,
 *                        batch): *s = 0 and *q = 0 when there is none
 * Return PM_OK, or PM_ERR_INVALID_ARG (null or empty path, a file that cannot
 * be written or read, a malformed file, an unknown form).
 */
#define PM_TUNE_PLAIN 1
#define PM_TUNE_BATCHED 2
pm_status polymul_tune_save(const char *path);
pm_status polymul_tune_load(const char *path);
pm_status polymul_tune_clear(void);
pm_status polymul_tune_lookup(const char *device, int sms, int form, uint32_t p, int64_t x, int64_t y, int *s,
                              int64_t *q);

/*
 * polymul_probe_mac_rate - measures the ceiling of the plain path: how many
 * 32 x 32 -> 64-bit multiply-adds (one per modular MAC of the s-blocked
 * product, Section 5's multiplication phase) an SM issues per clock.  Runs
 * blocks_per_sm x (SM count) blocks of `threads` threads, each thread adding
 * 16 independent products per iteration for `iters` iterations, and reads
 * every SM's cycle counter around its blocks' loops: the result, written to
 * *macs_per_clk_sm, is the mean over the SMs of products per clock, so it
 * does not depend on the clock.  Allocates (and frees) a small buffer;
 * synchronises `stream`.
 * Returns PM_OK, PM_ERR_INVALID_ARG (threads not a multiple of 32 in
 * [32, 1024], blocks_per_sm outside [1, 32], iters outside [4, 2^32]; iters is
 * rounded down to a multiple of 4), PM_ERR_UNSUPPORTED
 * (the stream captures), PM_ERR_NOMEM, PM_ERR_CUDA or PM_ERR_INTERNAL.
 */
pm_status polymul_probe_mac_rate(int threads, int blocks_per_sm, int64_t iters, double *macs_per_clk_sm,
                                 void *stream);

/*
 * polymul_tensor_limbs - the limb encoding of the tensor-core form
 * (polymul_batched with PM_TENSOR): a's coefficients, moved to the centred
 * range (-p/2, p/2], are written as *na balanced base-*base_a digits in
 * [-base_a/2, base_a/2), b's as *nb balanced base-*base_b digits; bf16 holds
 * every digit exactly, and an fp32 accumulator entry sums at most *max_terms
 * digit products, so its sums stay below 2^24 and exact (products whose
 * shorter operand is longer run in K-groups of max_terms / 32 shifts).  One
 * modular multiply-add costs na * nb bf16 limb products.  *tile_blocks is the
 * tile width in blocks of 32 outputs (every MMA spans it: 128 rows by
 * tile_blocks * na columns, two MMAs of K = 16 per shift of a tile).  Host
 * only; no GPU needed.  Returns PM_OK or PM_ERR_INVALID_ARG (a null pointer).
 */
pm_status polymul_tensor_limbs(int *na, int *nb, uint32_t *base_a, uint32_t *base_b, int *max_terms,
                               int *tile_blocks);

/*
 * polymul_probe_mma - measures one tcgen05 MMA kind on this device, for the
 * limb encodings of the tensor-core form (PM_TENSOR): kind PM_MMA_BF16 is
 * kind::f16 with bf16 operands (K = 16), the one the product kernel issues;
 * PM_MMA_E4M3 is kind::f8f6f4 with e4m3 operands (K = 32), which an
 * encoding in 4- or 5-bit limbs would issue.  One block per SM allocates 256
 * columns of tensor memory and, from constant operands in shared memory:
 * (1) accumulates a sum near 2^23 with full-width MMAs and then small
 * addends, an integer below 2^24, and checks 4 columns of all 128 lanes
 * against it: *exact = 1 if every entry of every SM equals it (the fp32
 * accumulation kept every bit), else 0; (2) issues `iters` full-width MMAs
 * (M = 128, N = 256) back to back and reads the SM's cycle counter from the
 * first issue to their completion: *flops_per_clk_sm is the mean over the
 * SMs of 2 M N K iters over those cycles (dense flops per clock per SM, not
 * dependent on the clock).  Synchronises `stream`; allocates (and frees) a
 * small buffer.
 * Returns PM_OK, PM_ERR_INVALID_ARG (null output, unknown kind, iters outside
 * [1, 2^20]), PM_ERR_UNSUPPORTED (not an sm_100-family device, or the stream
 * captures), PM_ERR_TIMEOUT (a bounded wait of the probe ran out), PM_ERR_NOMEM
 * or PM_ERR_CUDA.
 */
#define PM_MMA_BF16 0
#define PM_MMA_E4M3 1
pm_status polymul_probe_mma(int kind, int64_t iters, double *flops_per_clk_sm, int *exact, void *stream);

/*
 * polymul_sync_status - synchronises `stream`, then returns and clears the
 * device status word of the current device (PM_OK if no kernel reported an
 * error since the last call).
 */
pm_status polymul_sync_status(void *stream);

/* Frees every workspace the library holds on every device it used. */
pm_status polymul_release(void);

/* Static text for a status code. */
const char *polymul_status_string(pm_status status);

/* The last cudaError_t seen by a call that returned PM_ERR_CUDA (0 if none). */
int polymul_last_cuda_error(void);

/* Kernel launches made by this process so far (every entry point counts its own). */
uint64_t polymul_launch_count(void);

/*
 * polymul_debug_set - test hooks for the failure paths (the paper has no
 * counterpart).  Process-wide; not for production use.
 *
 *   PM_DEBUG_FAIL_ALLOC     the next `value` device allocations the library
 *                           makes (workspace, scratch, transform tables) fail
 *                           as if cudaMalloc had run out of memory: the call
 *                           that needed one returns PM_ERR_NOMEM and changes
 *                           nothing; 0 turns the hook off.
 *   PM_DEBUG_TC_WAIT_LIMIT  polls before a wait of the tensor-core kernel
 *                           (polymul_batched, PM_TENSOR) is declared lost;
 *                           0 = the built-in limit (2^26 polls).  A wait that
 *                           runs out sets PM_ERR_TIMEOUT in the status word
 *                           and the kernel ends its work early (outputs of the
 *                           tiles it did not finish are left as they were);
 *                           with value = 1 or more, the first wait of every
 *                           role may already run out.  Whatever ran out, the
 *                           kernel waits for the tensor-core operations it
 *                           issued (with a limit of its own) before it frees
 *                           its tensor memory.
 * Returns PM_OK, or PM_ERR_INVALID_ARG for an unknown knob or value < 0.
 */
#define PM_DEBUG_FAIL_ALLOC 1
#define PM_DEBUG_TC_WAIT_LIMIT 2
pm_status polymul_debug_set(int knob, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* POLYMUL_H */
