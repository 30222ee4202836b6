"""Parity of the GPU division (Section 3, Algorithms 3-4) with the division oracle, every word."""
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


def _case(n, m, seed, p=P):
    """a with n terms, b with m terms, uniform in [0, p), b's leading coefficient nonzero."""
    a, b = inputs.poly_pair(n - 1, m - 1, seed, p)
    if b[-1] == 0:
        b[-1] = 1
    return a.astype(np.uint32), b.astype(np.uint32)


def _check(a, b, p=P, s=0):
    q, r = pm.divide(dev(a), dev(b), p=p, s=s)
    assert pm.sync_status() == 0
    wq, wr = oracle.divide(a, b, p)
    assert_equal(host(q), wq, f"q n={len(a)} m={len(b)} s={s}")
    assert_equal(host(r), wr, f"r n={len(a)} m={len(b)} s={s}")


@pytest.mark.parametrize("s", [1, 2, 3, 7, 32, 64, 100, 256])
def test_s_values(s):
    a, b = _case(1300, 517, 101 + s)
    _check(a, b, s=s)


@pytest.mark.parametrize("n,m", [(1, 1), (2, 1), (9, 1), (5, 5), (6, 5), (257, 1), (512, 511),
                                 (513, 2), (1024, 513), (3000, 2999), (4100, 600), (2049, 1025)])
def test_shapes(n, m):
    a, b = _case(n, m, 7 * n + m)
    _check(a, b, s=0)
    _check(a, b, s=5)


def test_large_pair_and_other_moduli():
    a, b = _case(32768, 16384, 13)
    _check(a, b, s=256)
    for p in (2, 65537, (1 << 30) - 35):  # a prime just below 2^30
        a2, b2 = _case(2000, 700, 17, p)
        _check(a2, b2, p=p, s=64)


def test_exact_quotient_and_repeated_calls():
    """b * q0 divided by b: q0 back and a zero remainder, twice on the same scratch."""
    rng = np.random.default_rng(5)
    b = rng.integers(0, P, 900).astype(np.uint32)
    b[-1] = 3
    q0 = rng.integers(0, P, 1500).astype(np.uint32)
    a = oracle.polymul(q0, b, P)
    for _ in range(2):
        q, r = pm.divide(dev(a), dev(b), s=128)
        assert pm.sync_status() == 0
        assert_equal(host(q), q0, "quotient")
        assert (host(r) == 0).all()


def test_leading_coefficient_without_inverse():
    a = np.arange(1, 20, dtype=np.uint32)
    b = np.array([1, 2, 3], np.uint32)  # lc 3, p = 9: no inverse
    pm.divide(dev(a), dev(b), p=9, s=4)
    assert pm.sync_status() == 1
    assert pm.sync_status() == 0
