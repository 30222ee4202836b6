"""The in-tree measurements of the hardware the kernels are bounded by.

* polymul_probe_mac_rate: the 32 x 32 -> 64-bit multiply-add issue rate per
  clock per SM (the plain path's ceiling); the hardware issues it at most at
  the 32-bit integer multiply-add rate, so the probe reads between 16 and 64.
* polymul_probe_mma: the tcgen05 MMA kinds of the limb encodings.  The bf16
  kind the tensor-core form issues must accumulate exactly in fp32 (its
  products are exact only if it does) and run at a plausible dense rate
  (the nominal 2.25 PFLOP/s over 152 SMs at 2.07 GHz is 7150 flops per clock
  per SM); the e4m3 kind is measured, and its exactness reported.
"""
import pytest

from paper_1402_0264_gb300 import polymul as pm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_mac_rate_is_plausible():
    r = pm.probe_mac_rate(threads=256, blocks_per_sm=4, iters=4000)
    assert 16.0 <= r <= 64.0


def test_bf16_mma_accumulates_exactly_at_a_dense_rate():
    rate, exact = pm.probe_mma(pm.PM_MMA_BF16, iters=2048)
    assert exact, "kind::f16 bf16 accumulation lost bits below 2^24"
    assert 2000.0 < rate < 20000.0
    assert pm.sync_status() == 0


def test_e4m3_mma_is_measured():
    rate, exact = pm.probe_mma(pm.PM_MMA_E4M3, iters=2048)
    assert rate > 0.0
    assert isinstance(exact, bool)
    assert pm.sync_status() == 0
