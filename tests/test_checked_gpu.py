"""The range-checked build (-DPOLYMUL_CHECKED): guarded indices in every kernel that record
PM_ERR_INTERNAL instead of faulting, and an input scan that reports words >= p as PM_ERR_RANGE.
The build is compiled here and exercised in a process of its own (tests/checked_cases.py)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(900)
def test_checked_build_small_cases_and_range_reports():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1402_0264_gb300 import build
    oracle.build()
    lib = build.build(checked=True)
    env = dict(os.environ, POLYMUL_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "checked build ok" in r.stdout
