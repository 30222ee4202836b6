"""The bench's model ratios for division (Section 3) and the gcd (Section 6) against the closed
forms the paper prints for them.  The paper substitutes l = Z/2 and s = Z/7 (division), and
l = Z/2, s = Z/6, m = n (gcd); under those substitutions the ratios T_1/T_s built from its N, L
and C must reduce to the printed R.  Also the bench's count of the tensor kernel's issued work,
against a brute-force enumeration of the shifts each tile meets.  Host arithmetic only."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_models", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


@pytest.mark.parametrize("Z", [14.0, 64.0, 700.0, 3584.0])
@pytest.mark.parametrize("U", [0.5, 5.9, 40.0])
@pytest.mark.parametrize("n,m", [(4096, 2048), (32768, 16384), (10**6, 3)])
def test_division_ratio_is_the_printed_R(bench, Z, U, n, m):
    """Section 3: R = (3 + 5U) Z / (3 (Z + 21 U)) with s = Z/7 (l = Z/2 cancels)."""
    got = bench.division_model_ratio(n, m, Z / 7, Z / 2, U)
    want = (3 + 5 * U) * Z / (3 * (Z + 21 * U))
    assert got == pytest.approx(want, rel=1e-12)


def test_division_ratio_threshold(bench):
    """The paper's reading: R > 1 exactly when Z > 12.6, whatever U."""
    for U in (0.3, 5.9, 100.0):
        assert bench.division_model_ratio(5000, 1000, 12.6 / 7, 6.3, U) == pytest.approx(1.0, rel=1e-12)
        assert bench.division_model_ratio(5000, 1000, 13.0 / 7, 6.5, U) > 1.0
        assert bench.division_model_ratio(5000, 1000, 12.0 / 7, 6.0, U) < 1.0


@pytest.mark.parametrize("Z", [12.0, 96.0, 1536.0])
@pytest.mark.parametrize("U", [0.5, 5.9, 40.0])
@pytest.mark.parametrize("n", [1000, 9000, 10**6])
def test_gcd_ratio_is_the_printed_R(bench, Z, U, n):
    """Section 6: R = (6n - 2 + Z)(3 + 5U) Z / ((18 n + Z)(Z + 16 U)) with m = n, l = Z/2, s = Z/6."""
    got = bench.gcd_model_ratio(n, n, Z / 6, Z / 2, U)
    want = (6 * n - 2 + Z) * (3 + 5 * U) * Z / ((18 * n + Z) * (Z + 16 * U))
    assert got == pytest.approx(want, rel=1e-12)


def test_gcd_ratio_limit_and_threshold(bench):
    """As n grows, R tends to (3 + 5U) Z / (3 (Z + 16 U)), which exceeds 1 exactly when Z > 9.6."""
    U = 5.9
    for Z in (9.6, 20.0, 600.0):
        limit = (3 + 5 * U) * Z / (3 * (Z + 16 * U))
        assert bench.gcd_model_ratio(10**12, 10**12, Z / 6, Z / 2, U) == pytest.approx(limit, rel=1e-9)
    assert (3 + 5 * U) * 9.6 / (3 * (9.6 + 16 * U)) == pytest.approx(1.0, rel=1e-12)


def _issued_shifts_by_enumeration(n, m, W):
    """Shifts the tensor kernel issues for one pair, by brute force: for every tile of W output
    blocks, every shift delta whose b digits (indices 32 delta - 31 .. 32 delta + 31) meet b and
    whose a block I - delta exists for some output block I of the tile."""
    if m > n:
        n, m = m, n
    na = (n + 31) // 32
    L = n + m - 1
    total = 0
    for I0 in range(0, (L + 31) // 32, W):
        for delta in range(-2, (m + 31) // 32 + 2):
            meets_b = 32 * delta - 31 <= m - 1 and 32 * delta + 31 >= 0
            meets_a = any(0 <= I - delta < na for I in range(I0, I0 + W))
            total += meets_b and meets_a
    return total


def test_tc_issued_flops_matches_enumeration(bench):
    import numpy as np
    enc = {"tile_blocks": 64, "na": 4}
    rng = np.random.default_rng(5)
    n = rng.integers(1, 9000, 40)
    m = rng.integers(1, 9000, 40)
    n[:4] = [1, 4096, 31, 2593]
    m[:4] = [1, 4096, 4097, 33]
    a_off = np.concatenate([[0], np.cumsum(n)])
    b_off = np.concatenate([[0], np.cumsum(m)])
    shifts = sum(_issued_shifts_by_enumeration(int(x), int(y), 64) for x, y in zip(n, m))
    per_shift = 2 * 2 * 128 * 16 * 64 * 4   # two MMAs of 128 x 256 x 16
    assert bench.tc_issued_flops(a_off, b_off, enc) == shifts * per_shift


def test_headline_useful_over_issued_is_two_thirds(bench):
    """1024 pairs of degree 4095 with 64-block tiles: 384 shifts per pair of 128 x 128 blocks, so
    the useful share of the issued products is 128 * 128 * 32 / (384 * 64 * 32) = 2/3."""
    import numpy as np
    enc = {"tile_blocks": 64, "na": 4}
    off = np.arange(0, 1025 * 4096, 4096, dtype=np.int64)
    issued = bench.tc_issued_flops(off, off, enc)
    useful = 1024 * 4096 * 4096 * 16 * 2
    assert useful / issued == pytest.approx(2 / 3, rel=1e-12)
