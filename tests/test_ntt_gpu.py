"""Parity of the transform path with the CPU oracle (and with the plain path)."""
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


def run(a, b, p=P, g=0):
    out = pm.ntt(dev(a), dev(b), p=p, g=g)
    assert pm.sync_status() == 0
    return host(out)


SHAPES = [(1, 1), (2, 1), (3, 3), (100, 29), (1024, 1024), (2048, 2049), (2049, 2048),
          (5000, 3000), (4097, 1), (8192, 1), (4096, 4096), (6000, 2193), (20000, 12289), (65537, 3)]


@pytest.mark.parametrize("n,m", SHAPES)
def test_shapes_against_oracle(n, m):
    a = inputs.uniform_mod(40 + n, 1, n, P)
    b = inputs.uniform_mod(40 + m, 2, m, P)
    want = oracle.polymul(a, b, P) if n * m <= 2**26 else oracle.ntt_polymul(a, b, P)
    assert_equal(run(a, b), want, f"{n}x{m}")


@pytest.mark.parametrize("logn", list(range(10, 23)))
def test_degree_sweep(logn):
    """Equal degrees 2^k - 1 for k = 10..22 (transform lengths 2^11..2^23)."""
    n = 1 << logn
    a, b = inputs.workload_ntt(deg=n - 1, seed=inputs.SEED_BASE + 40 + logn)
    got = run(a, b)
    assert_equal(got, oracle.ntt_polymul(a, b, P), f"deg 2^{logn}-1")


def test_ntt_workload_full_checks():
    """Degree 2^22 - 1: full CPU transform oracle, definition at sampled k, evaluation."""
    a, b = inputs.workload_ntt()
    got = run(a, b)
    assert_equal(got, oracle.ntt_polymul(a, b, P), "deg 2^22-1")
    L = 2 * len(a) - 1
    ks = [0, 1, 2, len(a) - 1, len(a), L - 1, L // 2] + list(inputs.uniform_mod(7, 3, 24, L).astype(int))
    for k in ks:
        assert got[k] == oracle.coeff(a, b, P, int(k)), k
    for r in inputs.uniform_mod(7, 4, 4, P):
        r = int(r)
        assert oracle.evaluate(got, P, r) == (oracle.evaluate(a, P, r) * oracle.evaluate(b, P, r)) % P


def test_matches_plain_and_worst_case():
    a = np.full(30000, P - 1, np.uint32)
    b = np.full(17000, P - 1, np.uint32)
    k = np.arange(46999)
    want = (np.minimum.reduce([k + 1, np.full_like(k, 30000), np.full_like(k, 17000), 46999 - k]) % P)
    assert_equal(run(a, b), want.astype(np.uint32), "all p-1")
    a = inputs.uniform_mod(9, 1, 9000, P)
    b = inputs.uniform_mod(9, 2, 7001, P)
    assert_equal(run(a, b), host(pm.plain(dev(a), dev(b))), "ntt vs plain")


def test_other_prime_with_generator():
    p, g = 998244353, 3  # 119 * 2^23 + 1
    a = inputs.uniform_mod(5, 1, 70000, p)
    b = inputs.uniform_mod(5, 2, 50000, p)
    assert_equal(run(a, b, p=p, g=g), oracle.ntt_polymul(a, b, p, g), "p=998244353")
    for n, m in [(5000, 3000), (2000, 2000), (100, 29)]:  # transforms of 8192, 4096 and 128 points
        a = inputs.uniform_mod(6, 1, n, p)
        b = inputs.uniform_mod(6, 2, m, p)
        assert_equal(run(a, b, p=p, g=g), oracle.polymul(a, b, p), f"p=998244353 {n}x{m}")


@pytest.mark.parametrize("p,g", [(7681, 17), (12289, 11)])
def test_small_products_with_primes_of_low_two_adic_order(p, g):
    """7681 = 15 * 2^9 + 1 admits transforms up to length 512 only (the length-N transform in
    shared memory); 12289 = 3 * 2^12 + 1 exactly the length-4096 row transform, which products of
    1024 to 4096 points take."""
    top = (p - 1) & -(p - 1)
    for n, m in [(1, 1), (100, 29), (top // 2, top // 2), (top - 5, 6), (3, top - 2)]:
        a = inputs.uniform_mod(60 + n, 1, n, p)
        b = inputs.uniform_mod(60 + m, 2, m, p)
        assert_equal(run(a, b, p=p, g=g), oracle.polymul(a, b, p), f"p={p} {n}x{m}")
    with pytest.raises(pm.PolymulError) as e:
        pm.ntt(dev(np.ones(top, np.uint32)), dev(np.ones(2, np.uint32)), p=p, g=g)
    assert e.value.code == 3                # the product needs a transform of length 2 top


def test_unsupported_cases():
    a = dev(np.ones(70000, np.uint32))
    with pytest.raises(pm.PolymulError) as e:
        pm.ntt(a, a, p=65537, g=3)          # 2^18 does not divide 65536
    assert e.value.code == 3
    with pytest.raises(pm.PolymulError) as e:
        pm.ntt(dev(np.ones(10, np.uint32)), dev(np.ones(10, np.uint32)), p=998244353, g=0)
    assert e.value.code == 3                # no default generator for this prime
    with pytest.raises(pm.PolymulError) as e:
        pm.ntt(dev(np.ones(10, np.uint32)), dev(np.ones(10, np.uint32)), p=998244353, g=2)
    assert e.value.code == 3                # 2 has the wrong order: no root of order 32
