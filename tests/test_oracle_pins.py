"""Pins for the CPU oracle: facts fixed by mathematics, not by the oracle itself.

The oracle computes the long-multiplication product of Section 5
(f[k] = sum_{i+j=k} a[i] b[j] mod p).  Each test below checks it against
something independent, chosen so that a dropped term, a shifted index, a
wrong modulus or a swapped operand fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1402_0264_gb300 import inputs
from tests.refs import horner, kronecker_product

P = inputs.P_DEFAULT
P30 = 1073741789  # 2^30 - 35, prime (checked below)


# ---- Kronecker substitution: exact big-integer product, a different algorithm ----

@pytest.mark.parametrize("n,m", [(1, 1), (1, 5), (5, 1), (2, 3), (17, 64), (255, 256),
                                 (1000, 37), (1024, 1024), (2047, 1500)])
@pytest.mark.parametrize("p", [P, P30, 65537])
def test_matches_kronecker(n, m, p):
    a = inputs.uniform_mod(99 + n, 1, n, p)
    b = inputs.uniform_mod(99 + m, 2, m, p)
    np.testing.assert_array_equal(oracle.polymul(a, b, p), kronecker_product(a, b, p))


def test_unreduced_inputs_follow_definition():
    # the definition reduces sums, not inputs: values >= p must still give sum a_i b_j mod p
    rng = np.random.default_rng(5)
    a = rng.integers(0, 2**32, 300, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, 2**32, 301, dtype=np.uint64).astype(np.uint32)
    np.testing.assert_array_equal(oracle.polymul(a, b, P), kronecker_product(a, b, P))


# ---- brute force: every pair of short polynomials over small fields ----

def _all_polys(p, terms):
    return np.array(list(itertools.product(range(p), repeat=terms)), dtype=np.uint32)


@pytest.mark.parametrize("p,terms", [(7, 3), (17, 2), (5, 3)])
def test_exhaustive_small_field(p, terms):
    """f(x) = a(x) b(x) at every x in F_p; deg f < p, so this fixes f uniquely."""
    polys = _all_polys(p, terms)
    A = np.repeat(polys, len(polys), axis=0)
    B = np.tile(polys, (len(polys), 1))
    batch = len(A)
    off = np.arange(batch + 1, dtype=np.int64) * terms
    c_off = np.arange(batch + 1, dtype=np.int64) * (2 * terms - 1)
    F = oracle.polymul_batch(A.ravel(), off, B.ravel(), off, c_off, p).reshape(batch, 2 * terms - 1)
    assert 2 * terms - 2 < p
    xs = np.arange(p, dtype=np.int64)
    # evaluate all polynomials at all points with integer matrix products (Vandermonde)
    V = np.array([[pow(int(x), k, p) for k in range(2 * terms - 1)] for x in xs], dtype=np.int64)
    fa = (A.astype(np.int64) @ V[:, :terms].T) % p
    fb = (B.astype(np.int64) @ V[:, :terms].T) % p
    ff = (F.astype(np.int64) @ V.T) % p
    np.testing.assert_array_equal(ff, (fa * fb) % p)
    assert (F < p).all()


# ---- closed forms ----

@pytest.mark.parametrize("u,v", [(0, 0), (1, 1), (5, 9), (300, 1000), (2047, 2048)])
def test_binomial(u, v):
    """(1+x)^u (1+x)^v = (1+x)^(u+v): coefficients are binomials mod p."""
    a = np.array([math.comb(u, k) % P for k in range(u + 1)], dtype=np.uint32)
    b = np.array([math.comb(v, k) % P for k in range(v + 1)], dtype=np.uint32)
    want = np.array([math.comb(u + v, k) % P for k in range(u + v + 1)], dtype=np.uint32)
    np.testing.assert_array_equal(oracle.polymul(a, b, P), want)


@pytest.mark.parametrize("i,j,c1,c2", [(0, 0, 3, 5), (7, 0, P - 1, P - 1), (0, 9, 12345, 2),
                                       (100, 33, 469000000, 400000000)])
def test_monomials(i, j, c1, c2):
    a = np.zeros(i + 1, dtype=np.uint32); a[i] = c1
    b = np.zeros(j + 1, dtype=np.uint32); b[j] = c2
    want = np.zeros(i + j + 1, dtype=np.uint32); want[i + j] = (c1 * c2) % P
    np.testing.assert_array_equal(oracle.polymul(a, b, P), want)


def _trapezoid(n, m):
    k = np.arange(n + m - 1)
    return np.minimum.reduce([k + 1, np.full_like(k, n), np.full_like(k, m), n + m - 1 - k])


@pytest.mark.parametrize("n,m", [(1, 1), (1, 7), (8, 3), (1024, 1024), (4096, 33)])
def test_all_ones_and_all_minus_one(n, m):
    """(sum x^i)(sum x^j) has coefficient min(k+1, n, m, n+m-1-k); (p-1)^2 = 1 mod p too."""
    want = (_trapezoid(n, m) % P).astype(np.uint32)
    np.testing.assert_array_equal(oracle.polymul(np.ones(n, np.uint32), np.ones(m, np.uint32), P), want)
    a = np.full(n, P - 1, dtype=np.uint32)
    b = np.full(m, P - 1, dtype=np.uint32)
    np.testing.assert_array_equal(oracle.polymul(a, b, P), want)


# ---- identities ----

def test_identities():
    a = inputs.uniform_mod(7, 1, 333, P)
    b = inputs.uniform_mod(7, 2, 200, P)
    d = inputs.uniform_mod(7, 3, 200, P)
    ab = oracle.polymul(a, b, P)
    np.testing.assert_array_equal(ab, oracle.polymul(b, a, P))            # commutative
    bd = ((b.astype(np.uint64) + d) % P).astype(np.uint32)
    lhs = oracle.polymul(a, bd, P)
    rhs = ((ab.astype(np.uint64) + oracle.polymul(a, d, P)) % P).astype(np.uint32)
    np.testing.assert_array_equal(lhs, rhs)                                # distributive
    np.testing.assert_array_equal(oracle.polymul(a, np.ones(1, np.uint32), P), a)  # a*1 = a
    np.testing.assert_array_equal(oracle.polymul(a, np.zeros(5, np.uint32), P),
                                  np.zeros(337, np.uint32))                 # a*0 = 0 (with length kept)
    assert oracle.polymul(np.array([P - 2], np.uint32), np.array([3], np.uint32), P)[0] == (3 * (P - 2)) % P


def test_schwartz_zippel():
    a = inputs.uniform_mod(11, 1, 5000, P)
    b = inputs.uniform_mod(11, 2, 4321, P)
    f = oracle.polymul(a, b, P)
    for r in inputs.uniform_mod(11, 9, 8, P):
        r = int(r)
        assert horner(f, r, P) == (horner(a, r, P) * horner(b, r, P)) % P
        assert oracle.evaluate(f, P, r) == horner(f, r, P)


def test_coeff_matches_full_product():
    a = inputs.uniform_mod(13, 1, 700, P)
    b = inputs.uniform_mod(13, 2, 900, P)
    f = oracle.polymul(a, b, P)
    for k in [0, 1, 2, 699, 899, 1598, 800, 1234]:
        assert oracle.coeff(a, b, P, k) == f[k]


# ---- the transform-based evaluator, pinned to the definition ----

@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (3, 3), (100, 29), (1024, 1024), (1025, 1024),
                                 (4096, 4096), (5000, 3000)])
def test_ntt_oracle_matches_definition(n, m):
    a = inputs.uniform_mod(21 + n, 1, n, P)
    b = inputs.uniform_mod(21 + m, 2, m, P)
    np.testing.assert_array_equal(oracle.ntt_polymul(a, b, P), oracle.polymul(a, b, P))


def test_ntt_oracle_matches_kronecker_large():
    a = inputs.uniform_mod(3, 1, 20000, P)
    b = inputs.uniform_mod(3, 2, 12289, P)
    np.testing.assert_array_equal(oracle.ntt_polymul(a, b, P), kronecker_product(a, b, P))


def test_ntt_oracle_other_prime():
    p, g = 998244353, 3  # 119 * 2^23 + 1, generator 3
    a = inputs.uniform_mod(4, 1, 3000, p)
    b = inputs.uniform_mod(4, 2, 2000, p)
    np.testing.assert_array_equal(oracle.ntt_polymul(a, b, p, g), kronecker_product(a, b, p))


def test_ntt_oracle_rejects_unsupported_length():
    # 65537 - 1 = 2^16: a length-2^17 transform does not exist
    a = np.ones(70000, np.uint32)
    with pytest.raises(ValueError):
        oracle.ntt_polymul(a, a, 65537)


# ---- facts about the prime ----

def test_prime_facts():
    assert P == 7 * 2**26 + 1
    assert all(P30 % q for q in range(2, math.isqrt(P30) + 1))
    r = int(math.isqrt(P))
    assert all(P % q for q in range(2, r + 1)), "p must be prime"
    # 3 generates (Z/p)^*: its order divides 7*2^26 and is not a divisor of (p-1)/2 or (p-1)/7
    assert oracle.powmod(3, (P - 1) // 2, P) == P - 1
    assert oracle.powmod(3, (P - 1) // 7, P) != 1
    for k in range(1, 27):
        w = oracle.powmod(3, (P - 1) >> k, P)
        assert oracle.powmod(w, 1 << (k - 1), P) == P - 1   # order exactly 2^k
    assert pow(3, (P - 1) // 2, P) == P - 1                  # Python's pow agrees


# ---- the pins have teeth: a planted mistake in a CPU copy of the definition fails ----

def _definition_with_dropped_term(a, b, p):
    n, m = len(a), len(b)
    f = np.zeros(n + m - 1, dtype=np.uint64)
    for k in range(n + m - 1):
        lo, hi = max(0, k - m + 1), min(k, n - 1)
        s = 0
        for i in range(lo, hi):  # planted: hi is excluded
            s += int(a[i]) * int(b[k - i])
        f[k] = s % p
    return f.astype(np.uint32)


def test_planted_mistake_is_caught():
    n = m = 16
    want = (_trapezoid(n, m) % P).astype(np.uint32)
    got = _definition_with_dropped_term(np.ones(n, np.uint32), np.ones(m, np.uint32), P)
    assert not np.array_equal(got, want)


def test_multicore_timing_variants_equal_the_definition():
    """The OpenMP variants timed as the CPU baseline are the pinned definition shared out over
    threads: word-for-word equal to the single-thread oracle on ragged pairs and batches."""
    from paper_1402_0264_gb300 import inputs as _inp
    for da, db in ((0, 0), (1, 700), (2999, 1999), (4095, 4095)):
        a, b = _inp.poly_pair(da, db, 7000 + da)
        assert np.array_equal(oracle.polymul_omp(a, b, P), oracle.polymul(a, b, P))
    pk = _inp.workload_batched(batch=40)
    assert np.array_equal(oracle.polymul_batch_omp(*pk[:4], pk[4], P),
                          oracle.polymul_batch(*pk[:4], pk[4], P))
    assert oracle.omp_threads() >= 1
