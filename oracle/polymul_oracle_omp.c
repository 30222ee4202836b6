/*
 * Multi-core timing variants of the CPU oracle.  TEST INFRASTRUCTURE ONLY,
 * used for the CPU baseline of the bench (the oracle timed on all host
 * cores), never by the library.
 *
 * These compute nothing of their own: each output coefficient (or each pair
 * of a batch) is the pinned single-thread definition of polymul_oracle.c
 * (oracle_coeff, oracle_polymul: the long multiplication of Section 5),
 * shared out over OpenMP threads.  A CPU test checks that they equal the
 * single-thread oracle word for word.  Without OpenMP they run on one thread.
 */
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

uint32_t oracle_coeff(const uint32_t *a, int64_t n, const uint32_t *b, int64_t m, uint32_t p, int64_t k);
int oracle_polymul(const uint32_t *a, int64_t n, const uint32_t *b, int64_t m, uint32_t p, uint32_t *f);

/* Threads the variants below use (omp_get_max_threads(), 1 without OpenMP). */
int oracle_omp_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* f = a*b mod p, the coefficients f[k] shared out over the threads. */
int oracle_polymul_omp(const uint32_t *a, int64_t n, const uint32_t *b, int64_t m, uint32_t p, uint32_t *f) {
    if (n < 1 || m < 1 || p < 2) return -1;
    const int64_t L = n + m - 1;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t k = 0; k < L; ++k) f[k] = oracle_coeff(a, n, b, m, p, k);
    return 0;
}

/* A CSR batch, the pairs shared out over the threads (largest first is not
   needed: the schedule is dynamic with one pair per claim). */
int oracle_polymul_batch_omp(int64_t batch, const uint32_t *a, const int64_t *a_off, const uint32_t *b,
                             const int64_t *b_off, uint32_t *f, const int64_t *f_off, uint32_t p) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t i = 0; i < batch; ++i) {
        const int64_t n = a_off[i + 1] - a_off[i];
        const int64_t m = b_off[i + 1] - b_off[i];
        if (f_off[i + 1] - f_off[i] != n + m - 1 ||
            oracle_polymul(a + a_off[i], n, b + b_off[i], m, p, f + f_off[i]) != 0)
            bad |= 1;
    }
    return bad ? -1 : 0;
}
