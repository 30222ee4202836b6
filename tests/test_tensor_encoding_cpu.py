"""CPU checks of the tensor-core form's limb encoding as the library reports it
(polymul_tensor_limbs, host code): every centred residue of a prime below 2^29 has balanced
digits of the reported bases and counts, bf16 holds every digit exactly, max_terms digit
products stay within fp32's exact integers in any order of summation, and the epilogue's
limb recombination fits int64.  No kernel runs here."""
import numpy as np
import pytest

from paper_1402_0264_gb300 import build as pbuild
from paper_1402_0264_gb300 import polymul as pm

TC_MAX_P = 1 << 29   # the tensor-core form takes p < 2^29


@pytest.fixture(scope="module")
def enc():
    pbuild.build()
    return pm.tensor_limbs()


def balanced_digits(v, base, limbs):
    """Digits d_i in [-base/2, base/2) with v = sum d_i base^i, by the offset
    K = (base/2)(1 + base + ... + base^(limbs-1)): v + K in standard base-`base` digits."""
    k = (base // 2) * sum(base ** i for i in range(limbs))
    u = v + k
    assert 0 <= u < base ** limbs, (v, base, limbs)
    return [(u // base ** i) % base - base // 2 for i in range(limbs)]


def test_reported_shape(enc):
    assert enc["limb_products"] == enc["na"] * enc["nb"]
    assert enc["nb"] * 32 == 128                      # M = 128 rows: b's limbs x 32 offsets
    assert enc["tile_blocks"] % 16 == 0
    assert enc["tile_blocks"] * enc["na"] <= 256      # N of one MMA
    assert enc["max_terms"] % 32 == 0                 # K-groups of whole 32-term shifts


def test_digits_cover_every_centred_residue(enc):
    rng = np.random.default_rng(1402)
    lo, hi = -(TC_MAX_P // 2), TC_MAX_P // 2          # centred residues lie in (-p/2, p/2]
    vals = [lo, lo + 1, -1, 0, 1, hi - 1, hi] + [int(x) for x in rng.integers(lo, hi + 1, 4000)]
    for base, limbs in ((enc["base_a"], enc["na"]), (enc["base_b"], enc["nb"])):
        for v in vals:
            d = balanced_digits(v, base, limbs)
            assert all(-(base // 2) <= x < base // 2 for x in d)
            assert sum(x * base ** i for i, x in enumerate(d)) == v


def test_digits_are_exact_in_bf16(enc):
    torch = pytest.importorskip("torch")
    for base in (enc["base_a"], enc["base_b"]):
        x = torch.arange(-(base // 2), base // 2, dtype=torch.float32)
        assert torch.equal(x.to(torch.bfloat16).to(torch.float32), x)


def test_accumulation_stays_exact_in_fp32(enc):
    worst = (enc["base_a"] // 2) * (enc["base_b"] // 2)   # the largest digit product's magnitude
    bound = enc["max_terms"] * worst
    assert bound <= 1 << 24        # every partial sum, in any order, is an integer of at most 2^24
    # the extreme sums, accumulated in fp32 one term at a time, come out exact
    for sign in (1, -1):
        acc = np.float32(0)
        for _ in range(enc["max_terms"]):
            acc = np.float32(acc + np.float32(sign * worst))
        assert int(acc) == sign * bound
    # and max_terms is the largest whole number of 32-term shifts within the bound
    assert (enc["max_terms"] + 32) * worst > 1 << 24


def test_recombination_fits_int64(enc):
    """The epilogue forms sum_i base_a^i D_i over a's limbs in int64, each |D_i| <= 2^24."""
    s = sum(enc["base_a"] ** i for i in range(enc["na"]))
    assert (1 << 24) * s < (1 << 63)
