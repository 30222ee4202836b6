"""Parity of the GPU gcd (Section 6, Algorithms 10-11 with parameter s) with the gcd oracle, every word."""
import numpy as np
import pytest

import oracle
from paper_1402_0264_gb300 import inputs
from paper_1402_0264_gb300 import polymul as pm
from tests.gpuhelp import assert_equal, dev, host

pytestmark = pytest.mark.gpu
P = inputs.P_DEFAULT


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_0264_gb300 import build
    build.build()


def _check(a, b, p=P, s=0):
    a = np.asarray(a, dtype=np.uint32)
    b = np.asarray(b, dtype=np.uint32)
    n = max(len(a), len(b))
    out = dev(np.full(n, 0xFFFFFFFF, dtype=np.uint32))   # every word must be written
    g = pm.gcd(dev(a), dev(b), p=p, s=s, out=out)
    assert pm.sync_status() == 0
    want = oracle.gcd(a, b, p)
    assert_equal(host(g), want, f"gcd len(a)={len(a)} len(b)={len(b)} s={s} p={p}")
    full = host(out)
    assert not full[len(want):].any(), "words above the gcd's degree must be zero"
    return len(want) - 1


def _planted(dg, du, dw, seed, p=P):
    """b = g u, a = g (u w + 1): gcd exactly g (products by the oracle)."""
    g, u, w = inputs.gcd_factors(dg, du, dw, seed, p)
    v = oracle.polymul(u, w, p)
    v[0] = (int(v[0]) + 1) % p
    return oracle.polymul(g, v, p), oracle.polymul(g, u, p), g


@pytest.mark.parametrize("s", [1, 2, 3, 8, 31, 64, 128, 256])
def test_s_values(s):
    a, b, g = _planted(37, 700, 90, 11 + s)
    assert _check(a, b, s=s) == 37
    a2, b2 = inputs.poly_pair(900, 899, 300 + s)
    _check(a2, b2, s=s)


@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (1, 2), (5, 3), (33, 33), (256, 255), (257, 256),
                                 (513, 100), (1000, 999), (2049, 1500), (3001, 3001)])
def test_shapes_random(n, m):
    a, b = inputs.poly_pair(n - 1, m - 1, 7 * n + m)
    _check(a, b, s=0)
    _check(b, a, s=17)


@pytest.mark.parametrize("dg,du,dw", [(0, 300, 20), (1, 1, 1), (255, 256, 1), (256, 600, 300),
                                      (700, 1500, 5), (1200, 10, 10), (2500, 600, 600)])
def test_planted_gcd(dg, du, dw):
    a, b, g = _planted(dg, du, dw, dg + 3 * du + 5 * dw)
    assert _check(a, b, s=128) == dg
    assert _check(b, a, s=64) == dg
    if dg + du + dw < 1500:   # the naive gcd, one step per launch
        assert _check(a, b, s=1) == dg


@pytest.mark.parametrize("m,n", [(6, 4), (97, 89), (360, 240), (1024, 768), (3000, 1000), (4096, 4095)])
def test_cyclotomic_identity(m, n):
    def xk1(k):
        v = np.zeros(k + 1, np.uint32)
        v[0], v[k] = P - 1, 1
        return v

    import math
    assert _check(xk1(m), xk1(n), s=64) == math.gcd(m, n)


def test_sparse_inputs_large_degree_drops():
    """Mostly-zero polynomials: leading coefficients vanish in runs, rounds end early."""
    for seed in range(6):
        rng = np.random.default_rng(seed)
        n, m = 1500 + 97 * seed, 900 + 31 * seed
        a = (rng.integers(0, P, n) * (rng.random(n) < 0.03)).astype(np.uint32)
        b = (rng.integers(0, P, m) * (rng.random(m) < 0.05)).astype(np.uint32)
        a[-1], b[-1] = 5, 7
        for s in (8, 128):
            _check(a, b, s=s)
        # the same with a planted common factor x^k g
        g = np.zeros(41, np.uint32)
        g[40], g[3] = 1, 9
        _check(oracle.polymul(a, g, P), oracle.polymul(b, g, P), s=64)


def test_special_cases():
    rng = np.random.default_rng(1)
    a = rng.integers(0, P, 600).astype(np.uint32)
    a[-1] = 4242
    assert _check(a, np.zeros(3, np.uint32), s=64) == 599          # gcd(a, 0) = monic a
    assert _check(np.zeros(1, np.uint32), a, s=64) == 599
    assert _check(a, a, s=64) == 599                              # gcd(a, a)
    assert _check(np.zeros(5, np.uint32), np.zeros(9, np.uint32), s=8) == -1   # gcd(0, 0)
    assert _check(a, np.array([7], np.uint32), s=8) == 0          # nonzero constant
    assert _check(np.array([3], np.uint32), np.array([0], np.uint32), s=1) == 0
    padded = np.concatenate([a, np.zeros(300, np.uint32)])        # leading zeros (several heads)
    _check(padded, a[:400].copy(), s=32)
    _check(padded, np.concatenate([a[:100], np.zeros(600, np.uint32)]), s=256)
    # b divides a
    b = rng.integers(0, P, 300).astype(np.uint32)
    b[-1] = 1
    u = rng.integers(0, P, 777).astype(np.uint32)
    assert _check(oracle.polymul(b, u, P), b, s=128) == 299
    # words at or above p are taken mod p
    big = (a.astype(np.uint64) + P).astype(np.uint32)
    _check(big, b, s=64)


@pytest.mark.parametrize("p", [2, 3, 7, 65537, (1 << 30) - 35])
def test_other_primes(p):
    a, b = inputs.poly_pair(1200, 1100, 40 + p % 1000, p)
    _check(a, b, p=p, s=64)
    a2, b2, g = _planted(100, 500, 50, 41, p)
    _check(a2, b2, p=p, s=128)


def test_full_size_workload():
    """The bench's workload: a = g u of degree 9999, b = g v of degree 8999, gcd g of degree 1000."""
    g, u, v = inputs.workload_gcd()
    a, b = oracle.polymul(g, u, P), oracle.polymul(g, v, P)
    assert len(a) == 10000 and len(b) == 9000
    for s in (1, 32, 128, 256):
        assert _check(a, b, s=s) == 1000
    assert np.array_equal(host(pm.gcd(dev(a), dev(b), s=128)), g)


def test_side_stream():
    import torch
    a, b, g = _planted(50, 400, 40, 77)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ta, tb = dev(a), dev(b)
        out = pm.gcd(ta, tb, s=64, stream=st)
    st.synchronize()
    assert np.array_equal(host(out), g)


def test_non_invertible_leading_coefficient_sets_status():
    """Z/9Z is not a field: gcd(3x + 1, 0) needs 3^-1 mod 9, which does not exist."""
    pm.gcd(dev(np.array([1, 3], np.uint32)), dev(np.array([0], np.uint32)), p=9, s=4)
    assert pm.sync_status() == 1
    assert pm.sync_status() == 0   # reading the status clears it
