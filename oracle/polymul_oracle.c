/*
 * CPU oracle for dense univariate polynomial multiplication modulo a
 * word-size prime.  TEST INFRASTRUCTURE ONLY: the tests, the package's smoke
 * check and the CPU-baseline leg of the bench call this; the library never
 * does.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Haque, Moreno Maza, Xie, Section 5 "Polynomial
 * multiplication"): for a, b over the field K = Z/pZ with n and m terms
 * (deg a = n-1, deg b = m-1, terms counted "null or not" as in Section 3),
 * f = a * b is the long-multiplication result
 *     f[k] = sum_{i+j=k, 0<=i<n, 0<=j<m} a[i] * b[j]   (mod p),
 * k = 0 .. n+m-2.  Every GPU path of this project (the s-blocked plain
 * product of Algorithms 5-7, the batched form, the tensor-core form and the
 * NTT form) must reproduce these residues exactly.
 *
 * Functions:
 *   oracle_polymul            the definition above, one 128-bit running sum per k
 *   oracle_coeff              one f[k] by the same definition (spot checks)
 *   oracle_eval               Horner evaluation of a polynomial at a point
 *   oracle_ntt_polymul        the same product through a textbook radix-2
 *                             number-theoretic transform (Cooley-Tukey,
 *                             bit-reversal permutation first); only a faster
 *                             exact evaluator for sizes where the definition
 *                             is too slow, pinned against the definition
 *   oracle_powmod             modular exponentiation (square and multiply)
 *   oracle_invmod             modular inverse (extended Euclidean algorithm)
 *   oracle_divide             Euclidean division a = q b + r over Z/pZ
 *                             (Section 3, "Polynomial division": the division
 *                             steps of Algorithms 1-4, one leading
 *                             coefficient cancelled per step, done here one
 *                             step at a time)
 *   oracle_gcd                the monic greatest common divisor over Z/pZ
 *                             (Section 6, "Euclidean algorithm"), computed
 *                             here by the textbook remainder sequence
 *                             r_{i+1} = r_{i-1} mod r_i, then made monic
 *
 * Plain C, single threaded, unoptimised on purpose.
 */
#include <stdint.h>
#include <stdlib.h>

typedef unsigned __int128 u128;

static uint32_t mulmod(uint32_t x, uint32_t y, uint32_t p) {
    return (uint32_t)(((uint64_t)x * (uint64_t)y) % p);
}

uint32_t oracle_powmod(uint32_t base, uint64_t e, uint32_t p) {
    uint32_t r = 1 % p;
    uint32_t b = base % p;
    while (e) {
        if (e & 1) r = mulmod(r, b, p);
        b = mulmod(b, b, p);
        e >>= 1;
    }
    return r;
}

/* f[k] for one k, by the definition (Section 5, long multiplication). */
uint32_t oracle_coeff(const uint32_t *a, int64_t n, const uint32_t *b, int64_t m,
                      uint32_t p, int64_t k) {
    if (k < 0 || k > n + m - 2) return 0;
    int64_t ilo = k - (m - 1) > 0 ? k - (m - 1) : 0;
    int64_t ihi = k < n - 1 ? k : n - 1;
    u128 acc = 0;
    for (int64_t i = ilo; i <= ihi; ++i)
        acc += (u128)a[i] * (u128)b[k - i];
    return (uint32_t)(acc % p);
}

/* The full product f = a*b mod p; f has n+m-1 words.  Returns 0, or -1 on bad sizes. */
int oracle_polymul(const uint32_t *a, int64_t n, const uint32_t *b, int64_t m,
                   uint32_t p, uint32_t *f) {
    if (n < 1 || m < 1 || p < 2) return -1;
    for (int64_t k = 0; k <= n + m - 2; ++k)
        f[k] = oracle_coeff(a, n, b, m, p, k);
    return 0;
}

/* A batch in packed (CSR) form: pair i is a[a_off[i]..a_off[i+1]) etc. */
int oracle_polymul_batch(int64_t batch, const uint32_t *a, const int64_t *a_off,
                         const uint32_t *b, const int64_t *b_off,
                         uint32_t *f, const int64_t *f_off, uint32_t p) {
    for (int64_t i = 0; i < batch; ++i) {
        int64_t n = a_off[i + 1] - a_off[i];
        int64_t m = b_off[i + 1] - b_off[i];
        if (f_off[i + 1] - f_off[i] != n + m - 1) return -1;
        if (oracle_polymul(a + a_off[i], n, b + b_off[i], m, p, f + f_off[i]) != 0) return -1;
    }
    return 0;
}

/* Horner: poly(x) mod p for poly of len terms (index = degree). */
uint32_t oracle_eval(const uint32_t *poly, int64_t len, uint32_t p, uint32_t x) {
    uint64_t acc = 0;
    for (int64_t i = len - 1; i >= 0; --i)
        acc = ((acc * (uint64_t)(x % p)) + poly[i] % p) % p;
    return (uint32_t)acc;
}

/* ---- textbook radix-2 NTT (in place, bit-reversal first, then log2 N stages) ---- */

static void bit_reverse_permute(uint32_t *x, int64_t N) {
    for (int64_t i = 1, j = 0; i < N; ++i) {
        int64_t bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint32_t t = x[i]; x[i] = x[j]; x[j] = t; }
    }
}

/* y[k] = sum_j x[j] * w^(j*k) with w a primitive N-th root of unity mod p. */
static void ntt_inplace(uint32_t *x, int64_t N, uint32_t w, uint32_t p) {
    bit_reverse_permute(x, N);
    for (int64_t len = 2; len <= N; len <<= 1) {
        /* root of order len: w^(N/len) */
        uint32_t wl = oracle_powmod(w, (uint64_t)(N / len), p);
        for (int64_t start = 0; start < N; start += len) {
            uint32_t t = 1;
            for (int64_t j = 0; j < len / 2; ++j) {
                uint32_t u = x[start + j];
                uint32_t v = mulmod(x[start + j + len / 2], t, p);
                x[start + j] = (uint32_t)(((uint64_t)u + v) % p);
                x[start + j + len / 2] = (uint32_t)(((uint64_t)u + p - v) % p);
                t = mulmod(t, wl, p);
            }
        }
    }
}

/*
 * f = a*b mod p through length-N transforms, N the least power of two
 * >= n+m-1.  Needs 2^e | p-1 with N = 2^e and g a generator of (Z/p)^*.
 * Returns 0, -1 on bad sizes, -2 if p-1 is not divisible by N, -3 on no memory.
 */
int oracle_ntt_polymul(const uint32_t *a, int64_t n, const uint32_t *b, int64_t m,
                       uint32_t p, uint32_t g, uint32_t *f) {
    if (n < 1 || m < 1 || p < 3) return -1;
    int64_t L = n + m - 1, N = 1;
    while (N < L) N <<= 1;
    if ((uint64_t)(p - 1) % (uint64_t)N != 0) return -2;
    uint32_t *x = (uint32_t *)calloc((size_t)N, sizeof(uint32_t));
    uint32_t *y = (uint32_t *)calloc((size_t)N, sizeof(uint32_t));
    if (!x || !y) { free(x); free(y); return -3; }
    for (int64_t i = 0; i < n; ++i) x[i] = a[i] % p;
    for (int64_t i = 0; i < m; ++i) y[i] = b[i] % p;
    uint32_t w = oracle_powmod(g, (uint64_t)(p - 1) / (uint64_t)N, p);
    ntt_inplace(x, N, w, p);
    ntt_inplace(y, N, w, p);
    for (int64_t i = 0; i < N; ++i) x[i] = mulmod(x[i], y[i], p);
    /* inverse: transform with w^-1, then scale by N^-1 (Fermat inverses) */
    uint32_t winv = oracle_powmod(w, (uint64_t)p - 2, p);
    ntt_inplace(x, N, winv, p);
    uint32_t ninv = oracle_powmod((uint32_t)(N % p), (uint64_t)p - 2, p);
    for (int64_t i = 0; i < L; ++i) f[i] = mulmod(x[i], ninv, p);
    free(x);
    free(y);
    return 0;
}

/* Batch through the transform, pair by pair (same CSR layout as above). */
int oracle_ntt_polymul_batch(int64_t batch, const uint32_t *a, const int64_t *a_off,
                             const uint32_t *b, const int64_t *b_off,
                             uint32_t *f, const int64_t *f_off, uint32_t p, uint32_t g) {
    for (int64_t i = 0; i < batch; ++i) {
        int64_t n = a_off[i + 1] - a_off[i];
        int64_t m = b_off[i + 1] - b_off[i];
        if (f_off[i + 1] - f_off[i] != n + m - 1) return -1;
        int rc = oracle_ntt_polymul(a + a_off[i], n, b + b_off[i], m, p, g, f + f_off[i]);
        if (rc != 0) return rc;
    }
    return 0;
}

/* x^-1 mod p by the extended Euclidean algorithm; 0 when gcd(x, p) != 1. */
uint32_t oracle_invmod(uint32_t x, uint32_t p) {
    int64_t r0 = p, r1 = x % p, t0 = 0, t1 = 1;
    while (r1 != 0) {
        int64_t qt = r0 / r1, tmp;
        tmp = r0 - qt * r1; r0 = r1; r1 = tmp;
        tmp = t0 - qt * t1; t0 = t1; t1 = tmp;
    }
    if (r0 != 1) return 0;
    if (t0 < 0) t0 += p;
    return (uint32_t)t0;
}

/* Euclidean division over Z/pZ (Section 3): for a with n terms and b with m
 * terms, n >= m >= 1, the unique q (n-m+1 terms) and r (the low m-1 terms)
 * with a = q b + r and deg r < deg b.  The division steps run from the top,
 * i = n-1 down to m-1, as in Algorithm 1: the current coefficient a[i] gives
 * q[i-(m-1)] = a[i] lc(b)^-1, and that multiple of x^(i-(m-1)) b is
 * subtracted from the remainder (which cancels a[i]).  lc(b) = b[m-1] must
 * be invertible mod p.  Returns 0, -1 for bad sizes, -2 when b[m-1] has no
 * inverse, -3 when out of memory. */
int oracle_divide(const uint32_t *a, int64_t n, const uint32_t *b, int64_t m, uint32_t p,
                  uint32_t *q, uint32_t *r) {
    if (m < 1 || n < m) return -1;
    uint32_t inv = oracle_invmod(b[m - 1] % p, p);
    if (inv == 0) return -2;
    uint32_t *rem = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!rem) return -3;
    for (int64_t i = 0; i < n; ++i) rem[i] = a[i] % p;
    for (int64_t i = n - 1; i >= m - 1; --i) {
        uint32_t c = mulmod(rem[i], inv, p);
        q[i - (m - 1)] = c;
        for (int64_t j = 0; j < m; ++j) {
            uint32_t t = mulmod(c, b[j] % p, p);
            uint32_t *x = &rem[i - (m - 1) + j];
            *x = *x >= t ? *x - t : *x + p - t;
        }
    }
    for (int64_t i = 0; i < m - 1; ++i) r[i] = rem[i];
    free(rem);
    return 0;
}

/* Degree of x (terms 0..len-1) once its zero leading coefficients are
 * dropped; -1 for the zero polynomial. */
static int64_t true_degree(const uint32_t *x, int64_t len) {
    int64_t d = len - 1;
    while (d >= 0 && x[d] == 0) --d;
    return d;
}

/* The greatest common divisor of a (na terms) and b (nb terms) over
 * Z/pZ, p prime (Section 6): the Euclidean remainder sequence
 * r_0 = a, r_1 = b, r_{i+1} = r_{i-1} mod r_i until the remainder is
 * zero; the last nonzero r_i, divided by its leading coefficient, is the
 * gcd.  Leading zero coefficients of the inputs are allowed.  Writes the
 * monic gcd to g[0..deg] and its degree to *deg_g (-1 when a = b = 0, g
 * untouched then); g must hold max(na, nb) words.  Returns 0, -1 for bad
 * sizes, -2 when a leading coefficient has no inverse mod p, -3 when out of
 * memory. */
int oracle_gcd(const uint32_t *a, int64_t na, const uint32_t *b, int64_t nb, uint32_t p,
               uint32_t *g, int64_t *deg_g) {
    if (na < 0 || nb < 0) return -1;
    int64_t cap = (na > nb ? na : nb) + 1;
    uint32_t *u = (uint32_t *)calloc((size_t)cap, sizeof(uint32_t));
    uint32_t *v = (uint32_t *)calloc((size_t)cap, sizeof(uint32_t));
    if (!u || !v) { free(u); free(v); return -3; }
    for (int64_t i = 0; i < na; ++i) u[i] = a[i] % p;
    for (int64_t i = 0; i < nb; ++i) v[i] = b[i] % p;
    int64_t du = true_degree(u, na), dv = true_degree(v, nb);
    while (dv >= 0) {
        /* u <- u mod v: cancel the leading coefficient of u while deg u >= deg v */
        uint32_t inv = oracle_invmod(v[dv], p);
        if (inv == 0) { free(u); free(v); return -2; }
        while (du >= dv) {
            uint32_t c = mulmod(u[du], inv, p);
            int64_t shift = du - dv;
            for (int64_t j = 0; j <= dv; ++j) {
                uint32_t t = mulmod(c, v[j], p);
                uint32_t *x = &u[shift + j];
                *x = *x >= t ? *x - t : *x + p - t;
            }
            du = true_degree(u, du + 1);
        }
        /* (u, v) <- (v, u mod v) */
        uint32_t *w = u; u = v; v = w;
        int64_t dw = du; du = dv; dv = dw;
    }
    *deg_g = du;
    if (du >= 0) {
        uint32_t inv = oracle_invmod(u[du], p);
        if (inv == 0) { free(u); free(v); return -2; }
        for (int64_t i = 0; i <= du; ++i) g[i] = mulmod(u[i], inv, p);
    }
    free(u);
    free(v);
    return 0;
}
