"""Parity of the tensor-core batched form (bf16 limbs, fp32 accumulation) with the oracle."""
import numpy as np
import pytest

import oracle
from paper_1402_0264_gb300 import inputs
from paper_1402_0264_gb300 import polymul as pm
from tests.gpuhelp import assert_equal, dev, dev64, host

pytestmark = pytest.mark.gpu
P = inputs.P_DEFAULT


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_0264_gb300 import build
    build.build()


def run(packed, max_deg, p=P, mode=pm.PM_TENSOR):
    a_data, a_off, b_data, b_off, c_off = packed
    out = pm.batched(dev(a_data), dev64(a_off), dev(b_data), dev64(b_off), dev64(c_off),
                     max_deg=max_deg, p=p, mode=mode, total=int(c_off[-1]))
    assert pm.sync_status() == 0
    return host(out)


def test_small_ragged_batch():
    da = np.array([0, 1, 5, 31, 32, 33, 1000, 1535, 1536, 2047, 4095, 17, 1024, 2049, 2591], np.int64)
    db = np.array([0, 3, 5, 32, 31, 33, 17, 1536, 1535, 2047, 4095, 4000, 1025, 2048, 2592], np.int64)
    packed = inputs.packed_batch(da, db, 91)
    assert_equal(run(packed, 4095), oracle.polymul_batch(*packed[:4], packed[4], P))


@pytest.mark.parametrize("deg", [63, 1535, 3071, 4095])
def test_equal_degrees(deg):
    packed = inputs.workload_tensor(batch=16, deg=deg, seed=inputs.SEED_BASE + 300 + deg)
    assert_equal(run(packed, deg), oracle.polymul_batch(*packed[:4], packed[4], P), f"deg {deg}")


def test_random_unequal_pairs():
    """Degrees drawn independently in [0, 4095]: the per-shift column windows start and end
    at every offset within a tile."""
    rng = np.random.default_rng(1402)
    da = rng.integers(0, 4096, 96).astype(np.int64)
    db = rng.integers(0, 4096, 96).astype(np.int64)
    da[:4] = [4095, 0, 31, 4095]; db[:4] = [100, 4095, 4064, 32]
    packed = inputs.packed_batch(da, db, 92)
    assert_equal(run(packed, 4095), oracle.polymul_batch(*packed[:4], packed[4], P))


def _adversarial_values(p):
    """Coefficients whose balanced digits are all at the extreme -B/2 below the top limb (top limb
    0), for the encoding the library reports: every digit product is (B_a/2)(B_b/2), the largest
    the encoding has."""
    enc = pm.tensor_limbs()
    ba, bb = enc["base_a"], enc["base_b"]
    xa = p - (ba // 2) * sum(ba ** i for i in range(enc["na"] - 1))
    xb = p - (bb // 2) * sum(bb ** i for i in range(enc["nb"] - 1))
    return xa, xb


def _worst_case(deg, p=P):
    xa, xb = _adversarial_values(p)
    n = m = deg + 1
    a = np.full(n, xa, np.uint32)
    b = np.full(m, xb, np.uint32)
    a_off = np.array([0, n], np.int64); b_off = np.array([0, m], np.int64)
    c_off = np.array([0, n + m - 1], np.int64)
    return a, a_off, b, b_off, c_off


def test_adversarial_values_have_extreme_digits():
    """The values above: centred, they are -(B/2)(1 + B + ... + B^(L-2)), whose balanced digits are
    L-1 digits -B/2 and a top digit 0."""
    enc = pm.tensor_limbs()
    for x, base, limbs in zip(_adversarial_values(P), (enc["base_a"], enc["base_b"]), (enc["na"], enc["nb"])):
        v = int(x) - P
        u = v + (base // 2) * sum(base ** i for i in range(limbs))
        digits = [(u // base ** i) % base - base // 2 for i in range(limbs)]
        assert digits == [-(base // 2)] * (limbs - 1) + [0]
        assert 0 <= u < base ** limbs


def test_worst_case_accumulation():
    """Every digit product is the largest the encoding has and an entry meets max_terms of them in one
    accumulation (a pair of degree max_terms - 1, one K-group): the sums reach their bound (2^24 for
    the encoding of 5 base-64 by 4 base-256 limbs)."""
    deg = pm.tensor_limbs()["max_terms"] - 1
    a, a_off, b, b_off, c_off = _worst_case(deg)
    want = oracle.polymul(a, b, P)
    assert_equal(run((a, a_off, b, b_off, c_off), deg), want, "adversarial digits")
    # both operand orders, and all p-1
    assert_equal(run((b, b_off, a, a_off, c_off), deg), want, "swapped")
    ones = np.full(deg + 1, P - 1, np.uint32)
    assert_equal(run((ones, a_off, ones, b_off, c_off), deg), oracle.polymul(ones, ones, P), "p-1")


def test_worst_case_accumulation_degree_4095():
    """The headline degree with extreme digits (one K-group or several, by the encoding)."""
    a, a_off, b, b_off, c_off = _worst_case(4095)
    assert_equal(run((a, a_off, b, b_off, c_off), 4095), oracle.polymul(a, b, P), "adversarial digits")


@pytest.mark.parametrize("deg", [2592, 4096, 8191, 16383])
def test_degrees_beyond_one_k_group(deg):
    """Pairs whose operands both exceed max_terms terms (for some encoding): each tile is accumulated
    in K-groups of at most max_terms / 32 shifts and the groups' residues added in the epilogue."""
    packed = inputs.workload_tensor(batch=3, deg=deg, seed=inputs.SEED_BASE + 310 + deg)
    assert_equal(run(packed, deg), oracle.polymul_batch(*packed[:4], packed[4], P), f"deg {deg}")


def test_long_and_short_operands_beyond_4096():
    """Ragged pairs up to degree 16383: one or both operands beyond one K-group, both orders."""
    da = np.array([16383, 5000, 16383, 4096, 300, 12000, 0, 9000], np.int64)
    db = np.array([5000, 16383, 300, 4097, 16383, 12001, 16383, 8999], np.int64)
    packed = inputs.packed_batch(da, db, 93)
    assert_equal(run(packed, 16383), oracle.polymul_batch(*packed[:4], packed[4], P))


@pytest.mark.parametrize("deg", [8191, 16383])
def test_worst_case_accumulation_in_k_groups(deg):
    """Extreme digits at degrees 8191 and 16383: a K-group's sums reach their bound, and the groups
    of a tile are added mod p."""
    a, a_off, b, b_off, c_off = _worst_case(deg)
    n = m = deg + 1
    want = oracle.ntt_polymul(a, b, P)
    assert_equal(run((a, a_off, b, b_off, c_off), deg), want, "adversarial digits")
    assert_equal(run((b, b_off, a, a_off, c_off), deg), want, "swapped")
    k = np.array([0, 4095, 4096, 8191, n - 1, n + m - 2])
    assert_equal(want[k], [oracle.coeff(a, b, P, int(x)) for x in k], "transform oracle spot check")


def test_tensor_workload_full():
    """1024 pairs of degree 4095 against the transform oracle, plus the plain path."""
    packed = inputs.workload_tensor()
    got = run(packed, 4095)
    want = oracle.ntt_polymul_batch(*packed[:4], packed[4], P)
    assert_equal(got, want, "1024 x deg 4095")
    # a sample of pairs by the definition
    a_data, a_off, b_data, b_off, c_off = packed
    for i in (0, 511, 1023):
        a = a_data[a_off[i]:a_off[i + 1]]; b = b_data[b_off[i]:b_off[i + 1]]
        assert_equal(got[c_off[i]:c_off[i + 1]], oracle.polymul(a, b, P), f"pair {i}")


def test_matches_plain_batched_and_auto_mode():
    packed = inputs.workload_batched(batch=300)
    da = packed[1][1:] - packed[1][:-1]
    assert da.max() <= 2049
    t = run(packed, 2048, mode=pm.PM_TENSOR)
    pl = run(packed, 2048, mode=pm.PM_PLAIN)
    au = run(packed, 2048, mode=pm.PM_AUTO)     # degrees up to 2048: the plain form
    au4 = run(packed, 4095, mode=pm.PM_AUTO)    # a bound above 2048: the tensor form
    assert_equal(t, pl, "tensor vs plain")
    assert_equal(au, pl, "auto vs plain")
    assert_equal(au4, pl, "auto (tensor) vs plain")


def test_other_modulus():
    p = 65537
    packed = inputs.packed_batch(np.array([100, 4095]), np.array([4095, 3000]), 5, p)
    assert_equal(run(packed, 4095, p=p), oracle.polymul_batch(*packed[:4], packed[4], p))


def test_bad_offsets_and_degrees():
    import torch
    da = np.array([10, 5000], np.int64)
    packed = inputs.packed_batch(da, da, 3)
    out = torch.full((int(packed[4][-1]),), 7, dtype=torch.uint32, device="cuda")
    pm.batched(dev(packed[0]), dev64(packed[1]), dev(packed[2]), dev64(packed[3]), dev64(packed[4]),
               max_deg=4095, mode=pm.PM_TENSOR, out=out, total=out.numel())
    assert pm.sync_status() == 1   # a degree above max_deg is refused on the device
    assert (host(out) == 7).all()
