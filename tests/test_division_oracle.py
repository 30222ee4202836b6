"""Pins of the division oracle (Section 3: Euclidean division a = q b + r over Z/pZ).

Each check rests on something other than the oracle's own elimination loop:
exhaustive brute force in plain Python over a small field, the uniqueness of
(q, r) (a built as q0 b + r0 with the pinned product oracle must give back
exactly q0 and r0), the remainder theorem (division by x - c leaves a(c),
evaluated by Horner), and closed forms.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1402_0264_gb300 import inputs

P = inputs.P_DEFAULT


def _py_mul(x, y, p):
    out = [0] * (len(x) + len(y) - 1)
    for i, u in enumerate(x):
        for j, v in enumerate(y):
            out[i + j] = (out[i + j] + u * v) % p
    return out


def _py_add(x, y, p):
    n = max(len(x), len(y))
    x = list(x) + [0] * (n - len(x))
    y = list(y) + [0] * (n - len(y))
    return [(u + v) % p for u, v in zip(x, y)]


@pytest.mark.parametrize("p", [5, 7])
def test_exhaustive_small_field(p):
    """Every a of 1..4 terms and every b of 1..3 terms with a nonzero leading coefficient
    over Z/pZ: a == q b + r exactly, r has len(b) - 1 terms."""
    count = 0
    for m in (1, 2, 3):
        bs = [b for b in itertools.product(range(p), repeat=m) if b[-1] != 0]
        for n in range(m, 5):
            a_set = list(itertools.product(range(p), repeat=n))
            if len(a_set) * len(bs) > 60000:  # subsample the largest case deterministically
                a_set = a_set[::7]
            for a in a_set:
                for b in bs[:: max(1, len(bs) // 12)]:
                    q, r = oracle.divide(a, b, p)
                    assert len(q) == n - m + 1 and len(r) == m - 1
                    back = _py_add(_py_mul(list(q), list(b), p), list(r), p)
                    assert back[:n] == list(a) and all(v == 0 for v in back[n:]), (a, b, q, r)
                    count += 1
    assert count > 10000


@pytest.mark.parametrize("n,m", [(1, 1), (7, 1), (7, 7), (100, 37), (513, 256), (1000, 999)])
def test_uniqueness_against_the_product(n, m):
    """a = q0 b + r0 with deg r0 < deg b: the division returns q0 and r0 (the product is the
    pinned long-multiplication oracle)."""
    rng = np.random.default_rng(n * 1000 + m)
    q0 = rng.integers(0, P, n - m + 1).astype(np.uint32)
    b = rng.integers(0, P, m).astype(np.uint32)
    b[-1] = max(int(b[-1]), 1)
    r0 = rng.integers(0, P, m - 1).astype(np.uint32)
    a = oracle.polymul(q0, b, P).astype(np.uint64)
    a[: m - 1] = (a[: m - 1] + r0) % P
    q, r = oracle.divide(a.astype(np.uint32), b, P)
    assert np.array_equal(q, q0) and np.array_equal(r, r0)


def test_remainder_theorem():
    """Division by x - c leaves the value a(c) (Horner) and, for a = x^k, the quotient
    coefficients c^(k-1-j)."""
    rng = np.random.default_rng(3)
    for c in (0, 1, 2, P - 1, int(rng.integers(0, P))):
        a = rng.integers(0, P, 301).astype(np.uint32)
        _, r = oracle.divide(a, [(P - c) % P, 1], P)
        assert int(r[0]) == oracle.evaluate(a, P, c)
        k = 40
        xk = np.zeros(k + 1, np.uint32)
        xk[k] = 1
        q, r = oracle.divide(xk, [(P - c) % P, 1], P)
        assert [int(v) for v in q] == [oracle.powmod(c, k - 1 - j, P) for j in range(k)]
        assert int(r[0]) == oracle.powmod(c, k, P)


def test_closed_forms_and_edges():
    # (x^k - 1) / (x - 1) = 1 + x + ... + x^(k-1), no remainder
    for k in (1, 2, 17, 1000):
        a = np.zeros(k + 1, np.uint32)
        a[0], a[k] = P - 1, 1
        q, r = oracle.divide(a, [P - 1, 1], P)
        assert (q == 1).all() and len(q) == k and (r == 0).all()
    # constant divisor: q = a c^-1, no remainder
    a = np.arange(1, 50, dtype=np.uint32)
    q, r = oracle.divide(a, [5], P)
    inv5 = oracle.invmod(5, P)
    assert len(r) == 0 and [int(v) for v in q] == [(int(x) * inv5) % P for x in a]
    # equal degrees: one quotient term lc(a) / lc(b)
    q, r = oracle.divide([3, 4, 10], [1, 1, 5], P)
    assert list(q) == [2] and list(r) == [(3 - 2) % P, (4 - 2) % P]
    # b's leading coefficient without an inverse modulo a composite p
    with pytest.raises(ValueError):
        oracle.divide([1, 2, 3], [1, 6], 9)
    with pytest.raises(ValueError):
        oracle.divide([1], [1, 1], P)


def test_invmod():
    rng = np.random.default_rng(11)
    for x in list(rng.integers(1, P, 50)) + [1, 2, P - 1]:
        assert (int(x) * oracle.invmod(int(x), P)) % P == 1
    assert oracle.invmod(6, 9) == 0 and oracle.invmod(0, P) == 0
    assert (4 * oracle.invmod(4, 9)) % 9 == 1
