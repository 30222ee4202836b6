"""The bench's model ratios for division (Section 3) and the gcd (Section 6) against the closed
forms the paper prints for them.  The paper substitutes l = Z/2 and s = Z/7 (division), and
l = Z/2, s = Z/6, m = n (gcd); under those substitutions the ratios T_1/T_s built from its N, L
and C must reduce to the printed R.  Host arithmetic only."""
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
