"""The calibration of the model's U (Section 5's machine parameter) on measured times:
on times generated by the model itself with a known U and time scale, the fit recovers both."""
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_1402_0264_gb300 import polymul as pm  # noqa: E402

N = 16384
RATE, MHZ, P = 31.3, 2070.0, 152.0


def _points(U, kappa):
    pts = []
    for ell in (128, 256, 512):
        for s in pm.S_CANDIDATES:
            t = pm.model_predict(N, N, s, ell, U, P)["T_thm"] * ell / (RATE * MHZ * 1e6) * kappa
            pts.append((s, ell, t * 1e3))
    return pts


@pytest.mark.parametrize("U,kappa", [(2.0, 0.25), (5.9, 0.15), (16.0, 1.0)])
def test_fit_recovers_model_parameters(U, kappa):
    fit = bench.fit_model_U(pm.model_predict, _points(U, kappa), N, N, P, RATE, MHZ)
    assert abs(math.log2(fit["U_fit"] / U)) <= 1 / 32 + 1e-9  # the grid's half step
    assert fit["rms_log_err"] < 0.02
    assert abs(math.log(fit["kappa"] / kappa)) < 0.05
    for ell in (128, 256, 512):
        want = min(pm.S_CANDIDATES, key=lambda s: pm.model_predict(N, N, s, ell, U, P)["T_thm"])
        got = fit["best_s_fitted"][str(ell)]
        tw = pm.model_predict(N, N, want, ell, U, P)["T_thm"]
        tg = pm.model_predict(N, N, got, ell, U, P)["T_thm"]
        assert tg <= tw * 1.01


def test_fit_is_insensitive_to_a_time_scale():
    f1 = bench.fit_model_U(pm.model_predict, _points(4.0, 0.3), N, N, P, RATE, MHZ)
    f2 = bench.fit_model_U(pm.model_predict, _points(4.0, 3.0), N, N, P, RATE, MHZ)
    assert f1["U_fit"] == f2["U_fit"]
    assert abs(f2["kappa"] / f1["kappa"] - 10.0) < 1e-6
