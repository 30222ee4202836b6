"""The failure paths, driven on purpose without harming the GPU.

* An allocation failure is injected on the host (polymul_debug_set with
  PM_DEBUG_FAIL_ALLOC makes the library's next device allocation fail as if
  cudaMalloc had run out of memory): the call returns PM_ERR_NOMEM, writes
  nothing, and the next call on the same stream allocates and is correct.
* A bounded wait of the tensor-core kernel is made to run out: with a limit of
  one poll, the first wait between the kernel's roles that is not already
  complete gives up, the kernel records PM_ERR_TIMEOUT, ends its work early,
  waits for the tensor-core operations it issued, frees its tensor memory and
  returns; the context stays usable and the next call (default limit) is
  exact.
"""
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
    yield
    pm.debug_set(pm.PM_DEBUG_FAIL_ALLOC, 0)
    pm.debug_set(pm.PM_DEBUG_TC_WAIT_LIMIT, 0)


def test_injected_allocation_failure_returns_nomem():
    import torch
    a, b = inputs.poly_pair(3000, 2000, inputs.SEED_BASE + 600)
    ta, tb = dev(a), dev(b)
    pm.plain(ta, tb, s=8)  # the device workspace exists; the new stream below has no scratch yet
    st = torch.cuda.Stream()
    out = torch.full((len(a) + len(b) - 1,), 7, dtype=torch.uint32, device="cuda")
    pm.debug_set(pm.PM_DEBUG_FAIL_ALLOC, 1)
    with pytest.raises(pm.PolymulError) as ei:
        pm.plain(ta, tb, s=8, out=out, stream=st)
    assert ei.value.code == 4, ei.value  # PM_ERR_NOMEM
    st.synchronize()
    assert (host(out) == 7).all(), "a call that failed to allocate wrote output"
    # the hook fired once: the same call now allocates and is exact
    pm.plain(ta, tb, s=8, out=out, stream=st)
    st.synchronize()
    assert_equal(host(out), oracle.polymul(a, b, P), "after the injected failure")
    # the transform path (its tables or its scratch on this stream) fails the same way, then works
    a2, b2 = inputs.poly_pair(40000, 30000, inputs.SEED_BASE + 601)
    ta2, tb2 = dev(a2), dev(b2)
    pm.debug_set(pm.PM_DEBUG_FAIL_ALLOC, 1)
    with pytest.raises(pm.PolymulError) as ei:
        pm.ntt(ta2, tb2, stream=st)
    assert ei.value.code == 4
    got = pm.ntt(ta2, tb2, stream=st)
    st.synchronize()
    k = np.array([0, 1, 555, 40000, 70000], np.int64)
    want = [oracle.coeff(a2, b2, P, int(x)) for x in k]
    assert_equal(host(got)[k], want, "transform after the injected failure")
    assert pm.sync_status(st) == 0


def _tensor_batch():
    da = np.array([4095, 1000, 33, 2500], np.int64)
    db = np.array([4095, 3000, 4095, 7], np.int64)
    return inputs.packed_batch(da, db, inputs.SEED_BASE + 602)


def test_tensor_wait_that_runs_out_sets_timeout():
    import torch
    packed = _tensor_batch()
    t = [dev(packed[0]), dev64(packed[1]), dev(packed[2]), dev64(packed[3]), dev64(packed[4])]
    total = int(packed[4][-1])
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    out = torch.full((total,), 0xFFFFFFFF, dtype=torch.uint32, device="cuda")
    assert pm.sync_status() == 0
    pm.debug_set(pm.PM_DEBUG_TC_WAIT_LIMIT, 0)  # 0 = the default limit
    pm.batched(*t, max_deg=4095, mode=pm.PM_TENSOR, out=out, total=total)
    assert pm.sync_status() == 0
    assert_equal(host(out), want, "default limit")
    # a limit of one poll: the first wait that is not already complete runs out
    out.fill_(0xFFFFFFFF)
    pm.debug_set(pm.PM_DEBUG_TC_WAIT_LIMIT, 1)
    pm.batched(*t, max_deg=4095, mode=pm.PM_TENSOR, out=out, total=total)
    st = pm.sync_status()
    pm.debug_set(pm.PM_DEBUG_TC_WAIT_LIMIT, 0)
    assert st == 6, pm.STATUS.get(st, st)  # PM_ERR_TIMEOUT
    # the status word was cleared by the read; the next call is exact and clean
    out.fill_(0)
    pm.batched(*t, max_deg=4095, mode=pm.PM_TENSOR, out=out, total=total)
    assert pm.sync_status() == 0
    assert_equal(host(out), want, "after the timeout")


def test_debug_knob_rejects_unknown_values():
    assert pm.lib().polymul_debug_set(99, 1) == 1
    assert pm.lib().polymul_debug_set(pm.PM_DEBUG_FAIL_ALLOC, -1) == 1
