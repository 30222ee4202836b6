"""Pins for the fp64 cost model (Section 5 formulas, Theorem 1, Corollary 1).

The paper prints the per-s formulas (W_s, S_s, O_s, N_s, L_s, C_s) and,
separately, the ratios W_1/W_s, S_1/S_s, O_1/O_s (m = n) and the
Corollary-1 ratio R.  The ratios are consequences of the formulas, so
evaluating the oracle's formulas and dividing must give the printed ratios:
a typo in any single formula breaks one of these equalities.
"""
import json
import math
import os

import pytest

from oracle import model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

NS = [64, 1000, 4000, 8000, 16384, 2**20]
SS = [1, 2, 4, 8, 16, 32, 64]
US = [1.5, 4.0, 22.0, 400.0]
ELLS = [32, 128, 256]


def close(x, y, rel=1e-12):
    return math.isclose(x, y, rel_tol=rel, abs_tol=0.0)


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("s", SS)
def test_work_and_span_ratios(n, s):
    assert close(model.work(n, n, 1) / model.work(n, n, s), model.printed_work_ratio(n, s))
    assert close(model.span(n, n, 1) / model.span(n, n, s), model.printed_span_ratio(n, s))


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("s", SS)
@pytest.mark.parametrize("U", US)
@pytest.mark.parametrize("ell", ELLS)
def test_overhead_ratio(n, s, U, ell):
    r = model.overhead(n, n, 1, ell, U) / model.overhead(n, n, s, ell, U)
    assert close(r, model.printed_overhead_ratio(n, s))


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("s", SS)
@pytest.mark.parametrize("U", US)
@pytest.mark.parametrize("ell", ELLS)
def test_corollary1_ratio_is_printed_R(n, s, U, ell):
    """Corollary 1 with K = number of MulKer blocks reproduces the printed R."""
    r = model.corollary1(n, n, 1, ell, U) / model.corollary1(n, n, s, ell, U)
    assert close(r, model.printed_R(n, s, U), rel=1e-11)


def test_R_is_one_at_s1_and_below_one_above():
    for n in NS:
        for U in US:
            assert close(model.printed_R(n, 1, U), 1.0)
            for s in SS[1:]:
                assert model.printed_R(n, s, U) < 1.0   # "s = 1 performs better" (Section 5)


def test_overhead_ratio_limit():
    """As n grows, O_1/O_s -> 7 s^2 / (5 s + 2): Theta(s), the paper's "equivalent to s"."""
    for s in SS:
        lim = 7.0 * s * s / (5.0 * s + 2.0)
        assert abs(model.printed_overhead_ratio(1e13, s) / lim - 1.0) < 1e-9
        assert 0.9 * s <= lim <= 1.4 * s


def test_block_counts_and_levels():
    n = m = 16384
    for s in SS:
        for ell in ELLS:
            K = model.mulker_blocks(n, m, s, ell)
            assert close(K, (m / s) * (n + s - 1) / (s * ell))
            # the thread-block DAG holds the MulKer blocks plus the AddKer blocks
            assert model.blocks(n, m, s, ell) > K
        assert close(model.levels(m, s), math.log2(m // s) + 1)


def test_theorem1_dominates_corollary_when_P_small():
    # with P below the antichain width K, Theorem 1's N/P term is the larger one
    n = m = 8000
    for s in SS:
        K = model.mulker_blocks(n, m, s, 128)
        P = max(1.0, K / 4)
        assert model.theorem1(n, m, s, 128, 10.0, P) >= model.corollary1(n, m, s, 128, 10.0)


def test_local_memory_constraint():
    assert model.local_memory_ok(4, 256, 2 * 4 * 256 + 2 * 4 - 1)
    assert not model.local_memory_ok(4, 256, 2 * 4 * 256 + 2 * 4 - 2)


def test_table1_fixture_best_s_is_4():
    """Table 1 as transcribed: s = 4 is fastest on every row (Section 5, Conclusion)."""
    with open(os.path.join(GOLDEN, "table1_polymul_times.json")) as fh:
        t = json.load(fh)
    assert len(t["rows"]) == 9
    for row in t["rows"]:
        times = dict(zip(t["s"], row["seconds"]))
        assert min(times, key=times.get) == 4
