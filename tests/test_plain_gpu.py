"""Parity of the s-blocked plain product (Section 5, Algorithms 5-7) with the
CPU oracle, word for word, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1402_0264_gb300 import inputs
from paper_1402_0264_gb300 import polymul as pm
from tests.gpuhelp import assert_equal, dev, host

pytestmark = pytest.mark.gpu
P = inputs.P_DEFAULT
P30 = 1073741789
SS = [1, 2, 4, 8, 16, 32, 64]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_0264_gb300 import build
    build.build()


def run(a, b, p=P, s=0):
    out = pm.plain(dev(a), dev(b), p=p, s=s)
    assert pm.sync_status() == 0
    return host(out)


@pytest.mark.parametrize("s", SS)
def test_small_workload_all_s(s):
    a, b = inputs.workload_small()
    assert_equal(run(a, b, s=s), oracle.polymul(a, b, P), f"deg 1023, s={s}")


SHAPES = [(1, 1), (1, 5), (5, 1), (2, 3), (33, 17), (100, 1000), (1000, 100), (257, 256),
          (2049, 2047), (4097, 300), (5000, 7), (3000, 2900), (6001, 4099)]


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("s", SS)
def test_ragged_shapes(n, m, s):
    a = inputs.uniform_mod(1000 + n, 1, n, P)
    b = inputs.uniform_mod(2000 + m, 2, m, P)
    assert_equal(run(a, b, s=s), oracle.polymul(a, b, P), f"{n}x{m} s={s}")


@pytest.mark.parametrize("p", [2, 3, 65537, 998244353, P30])
@pytest.mark.parametrize("s", [1, 4, 8, 64])
def test_other_moduli(p, s):
    a = inputs.uniform_mod(5, 1, 3001, p)
    b = inputs.uniform_mod(5, 2, 2222, p)
    assert_equal(run(a, b, p=p, s=s), oracle.polymul(a, b, p), f"p={p} s={s}")


@pytest.mark.parametrize("s", SS)
def test_worst_case_accumulation(s):
    """All coefficients p-1 maximise every product; (p-1)^2 = 1 gives a trapezoid."""
    for p in (P, P30):
        n, m = 20000, 17000
        a = np.full(n, p - 1, np.uint32)
        b = np.full(m, p - 1, np.uint32)
        k = np.arange(n + m - 1)
        want = (np.minimum.reduce([k + 1, np.full_like(k, n), np.full_like(k, m), n + m - 1 - k]) % p)
        assert_equal(run(a, b, p=p, s=s), want.astype(np.uint32), f"p={p} s={s}")


def test_zero_and_monomials():
    z = np.zeros(100, np.uint32)
    a = inputs.uniform_mod(8, 1, 77, P)
    assert_equal(run(a, z), np.zeros(176, np.uint32))
    x = np.zeros(500, np.uint32); x[499] = P - 2
    y = np.zeros(300, np.uint32); y[0] = 3
    want = np.zeros(799, np.uint32); want[499] = (3 * (P - 2)) % P
    assert_equal(run(x, y), want)


@pytest.mark.parametrize("s", [0, 4, 8, 16])
def test_single_workload_full(s):
    """One pair of degree 16383, every output word against the oracle."""
    a, b = inputs.workload_single()
    assert_equal(run(a, b, s=s), oracle.polymul(a, b, P), f"deg 16383 s={s}")


def test_large_ragged_spot_checks():
    """deg 2^20 x 70000: sampled coefficients by definition, plus evaluation at random points."""
    n, m = 2**20 + 1, 70001
    a = inputs.uniform_mod(31, 1, n, P)
    b = inputs.uniform_mod(31, 2, m, P)
    got = run(a, b, s=8)
    ks = list(inputs.uniform_mod(31, 7, 48, n + m - 1).astype(np.int64)) + [0, 1, m - 1, n - 1, n + m - 2]
    for k in ks:
        assert got[k] == oracle.coeff(a, b, P, int(k)), k
    for r in inputs.uniform_mod(31, 8, 4, P):
        r = int(r)
        assert oracle.evaluate(got, P, r) == (oracle.evaluate(a, P, r) * oracle.evaluate(b, P, r)) % P


def test_commutative_and_stream_ordered():
    import torch
    a = inputs.uniform_mod(3, 1, 3000, P)
    b = inputs.uniform_mod(3, 2, 5000, P)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        da, db = dev(a), dev(b)
        c1 = pm.plain(da, db, s=8, stream=st)
        c2 = pm.plain(db, da, s=16, stream=st)
    st.synchronize()
    assert_equal(host(c1), host(c2))


def test_rejects_bad_arguments():
    a = dev(np.ones(10, np.uint32))
    with pytest.raises(pm.PolymulError):
        pm.plain(a, a, s=3)
    with pytest.raises(pm.PolymulError):
        pm.plain(a, a, p=2**30)
    with pytest.raises(TypeError):
        pm.plain(a.cpu(), a)


def test_tuner_picks_a_candidate():
    a, b = inputs.workload_single()
    best, times = pm.tune_plain(dev(a), dev(b), reps=2)
    assert best in SS and best in times
    assert pm.default_s(len(a) - 1, len(b) - 1) == best


@pytest.mark.parametrize("ell", [128, 512])
@pytest.mark.parametrize("s", [1, 4, 8, 32, 64])
def test_block_size_study(ell, s):
    """polymul_plain_ell: the same words as the oracle for l = 128 and 512 threads per block."""
    a, b = inputs.poly_pair(3000, 1700, inputs.SEED_BASE + 900 + s)
    got = host(pm.plain_ell(dev(a), dev(b), s=s, ell=ell))
    assert pm.sync_status() == 0
    assert_equal(got, oracle.polymul(a, b, P), f"l={ell} s={s}")
