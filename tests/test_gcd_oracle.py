"""Pins of the gcd oracle (Section 6: the Euclidean algorithm over Z/pZ).

Each check rests on something other than the oracle's remainder sequence:
exhaustive search for the monic common divisor of largest degree over small
fields, a gcd built in (a = g u, b = g (u w + 1), whose gcd is exactly g), the
identity gcd(x^m - 1, x^n - 1) = x^gcd(m, n) - 1, products of linear factors
whose common roots are known, and the special cases of the definition.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1402_0264_gb300 import inputs

P = inputs.P_DEFAULT


def _py_rem(x, y, p):
    """x mod y in plain Python (y monic-or-not, nonzero leading coefficient)."""
    x = list(x)
    dy = len(y) - 1
    inv = pow(y[-1], p - 2, p)
    for i in range(len(x) - 1, dy - 1, -1):
        c = x[i] * inv % p
        if c:
            for j in range(dy + 1):
                x[i - dy + j] = (x[i - dy + j] - c * y[j]) % p
    return x[:dy]


def _trim(x):
    x = list(x)
    while x and x[-1] == 0:
        x.pop()
    return x


def _py_mul(x, y, p):
    out = [0] * (len(x) + len(y) - 1)
    for i, u in enumerate(x):
        for j, v in enumerate(y):
            out[i + j] = (out[i + j] + u * v) % p
    return out


def _brute_gcd(a, b, p):
    """The monic common divisor of largest degree, by trying every monic polynomial."""
    a, b = _trim(a), _trim(b)
    if not a and not b:
        return []
    bound = min(len(x) for x in (a, b) if x) - 1
    for d in range(bound, -1, -1):
        for low in itertools.product(range(p), repeat=d):
            cand = list(low) + [1]
            if all(not _trim(_py_rem(x, cand, p)) for x in (a, b) if x):
                return cand
    raise AssertionError("1 divides everything")


@pytest.mark.parametrize("p,terms,stride", [(2, 5, 1), (3, 4, 1), (5, 3, 1), (7, 3, 5)])
def test_exhaustive_small_field(p, terms, stride):
    polys = list(itertools.product(range(p), repeat=terms))
    pairs = list(itertools.product(polys, polys))[::stride]
    for a, b in pairs[:: max(1, len(pairs) // 3000)]:
        want = _brute_gcd(a, b, p)
        got = [int(v) for v in oracle.gcd(a, b, p)]
        assert got == want, (a, b, got, want)


@pytest.mark.parametrize("dg,du,dw", [(0, 5, 3), (1, 1, 1), (7, 40, 9), (100, 150, 30), (500, 1200, 300)])
def test_constructed_gcd(dg, du, dw):
    """a = g u, b = g (u w + 1): gcd(u, u w + 1) = 1, so gcd(a, b) = g for monic g."""
    rng = np.random.default_rng(dg * 7 + du)
    g = rng.integers(0, P, dg + 1).astype(np.uint32)
    g[-1] = 1
    u = rng.integers(1, P, du + 1).astype(np.uint32)
    w = rng.integers(1, P, dw + 1).astype(np.uint32)
    v = oracle.polymul(u, w, P)
    v[0] = (int(v[0]) + 1) % P
    a, b = oracle.polymul(g, u, P), oracle.polymul(g, v, P)
    assert np.array_equal(oracle.gcd(a, b, P), g)
    assert np.array_equal(oracle.gcd(b, a, P), g)
    # a unit multiple of either argument leaves the gcd unchanged
    a7 = (a.astype(np.uint64) * 7 % P).astype(np.uint32)
    assert np.array_equal(oracle.gcd(a7, b, P), g)


@pytest.mark.parametrize("m,n", [(6, 4), (12, 18), (35, 21), (97, 89), (360, 240), (1024, 768)])
def test_cyclotomic_identity(m, n):
    """gcd(x^m - 1, x^n - 1) = x^gcd(m, n) - 1 over any field."""
    def xk1(k):
        v = np.zeros(k + 1, np.uint32)
        v[0], v[k] = P - 1, 1
        return v

    assert np.array_equal(oracle.gcd(xk1(m), xk1(n), P), xk1(math.gcd(m, n)))


def test_common_roots():
    """Products of distinct linear factors: the gcd is the product over the common roots."""
    rng = np.random.default_rng(5)
    pool = [int(x) for x in rng.choice(10**6, 60, replace=False)]
    for trial in range(6):
        ra = set(rng.choice(pool, 25, replace=False).tolist())
        rb = set(rng.choice(pool, 20, replace=False).tolist())

        def prod(roots):
            out = [1]
            for r in sorted(roots):
                out = _py_mul(out, [(P - r) % P, 1], P)
            return out

        want = prod(ra & rb)
        got = [int(v) for v in oracle.gcd(prod(ra), prod(rb), P)]
        assert got == want, trial


def test_special_cases():
    rng = np.random.default_rng(9)
    a = rng.integers(0, P, 50).astype(np.uint32)
    a[-1] = 12345
    inv = pow(12345, P - 2, P)
    monic_a = [int(x) * inv % P for x in a]
    assert [int(v) for v in oracle.gcd(a, [0, 0, 0], P)] == monic_a      # gcd(a, 0) = monic a
    assert [int(v) for v in oracle.gcd([0], a, P)] == monic_a
    assert [int(v) for v in oracle.gcd(a, a, P)] == monic_a              # gcd(a, a)
    assert len(oracle.gcd([0, 0], [0], P)) == 0                          # gcd(0, 0) = 0
    assert [int(v) for v in oracle.gcd(a, [5], P)] == [1]                # nonzero constant
    # leading zeros are ignored; with a(0) = 0 != a'(0), gcd(a, 3 x^2) = x
    z = np.concatenate([a, np.zeros(7, np.uint32)])
    z[0], z[1] = 0, 17
    assert [int(v) for v in oracle.gcd(z, [0, 0, 3, 0], P)] == [0, 1]
    z[1] = 0
    assert [int(v) for v in oracle.gcd(z, [0, 0, 3, 0], P)] == [0, 0, 1]


def test_workload_cofactors_are_coprime():
    """The gcd workloads plant g through a = g u, b = g v: their gcd is g only if gcd(u, v) = 1."""
    for seed_off, (dg, du, dv) in ((7, (1000, 8999, 7999)), (8, (200, 1799, 1299))):
        g, u, v = inputs.gcd_cofactors(dg, du, dv, inputs.SEED_BASE + seed_off)
        assert np.array_equal(oracle.gcd(u, v, P), [1])
        assert int(g[-1]) == 1 and len(g) == dg + 1
    g, u, v = inputs.workload_gcd()
    assert np.array_equal(oracle.gcd(oracle.polymul(g, u, P), oracle.polymul(g, v, P), P), g)
