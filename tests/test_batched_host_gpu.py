"""Parity of the host-buffer batched product (polymul_batched_host) with the CPU oracle and with
the device-buffer call: chunks, slot reuse across calls, pinned and pageable host arrays."""
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


def pinned(x):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.pin_memory()


def run_host(packed, max_deg, mode, pin=True, s=0):
    import torch
    a, a_off, b, b_off, c_off = packed
    conv = pinned if pin else np.ascontiguousarray
    arrays = [conv(np.asarray(a, np.uint32)), conv(np.asarray(a_off, np.int64)), conv(np.asarray(b, np.uint32)),
              conv(np.asarray(b_off, np.int64)), conv(np.asarray(c_off, np.int64))]
    out = conv(np.zeros(int(c_off[-1]), np.uint32))
    pm.batched_host(*arrays, out, max_deg=max_deg, mode=mode, s=s)
    torch.cuda.current_stream().synchronize()
    assert pm.sync_status() == 0
    return np.asarray(out.numpy() if hasattr(out, "numpy") else out).view(np.uint32).copy()


def run_dev(packed, max_deg, mode, s=0):
    a, a_off, b, b_off, c_off = packed
    out = pm.batched(dev(a), dev64(a_off), dev(b), dev64(b_off), dev64(c_off), max_deg=max_deg, mode=mode, s=s,
                     total=int(c_off[-1]))
    return host(out)


@pytest.mark.parametrize("mode", [pm.PM_TENSOR, pm.PM_PLAIN])
def test_equal_degrees_against_oracle(mode):
    packed = inputs.workload_tensor(batch=48, deg=4095, seed=inputs.SEED_BASE + 401)
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    assert_equal(run_host(packed, 4095, mode), want, f"mode {mode}")


def test_ragged_batch_against_oracle_pinned_and_pageable():
    rng = np.random.default_rng(1403)
    da = rng.integers(0, 2500, 61).astype(np.int64)
    db = rng.integers(0, 2500, 61).astype(np.int64)
    da[:3] = [0, 2499, 17]; db[:3] = [2499, 0, 3000 - 1 - 500]
    packed = inputs.packed_batch(da, db, 402)
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    for mode in (pm.PM_PLAIN, pm.PM_TENSOR, pm.PM_AUTO):
        assert_equal(run_host(packed, 2999, mode, pin=True), want, f"pinned, mode {mode}")
        assert_equal(run_host(packed, 2999, mode, pin=False), want, f"pageable, mode {mode}")


def test_small_batches_and_calls_in_a_row():
    """Fewer pairs than chunks, one pair, and successive calls of growing and shrinking size reusing
    the library's two chunk slots: each matches the device-buffer call word for word."""
    for k, (nb, deg) in enumerate([(1, 10), (2, 300), (3, 4095), (200, 1023), (5, 2047), (1, 4095)]):
        packed = inputs.workload_tensor(batch=nb, deg=deg, seed=inputs.SEED_BASE + 410 + k)
        want = run_dev(packed, deg, pm.PM_AUTO)
        assert_equal(run_host(packed, deg, pm.PM_AUTO), want, f"{nb} pairs of degree {deg}")
        assert_equal(run_host(packed, deg, pm.PM_AUTO), want, f"{nb} pairs of degree {deg}, again")


def test_headline_batch_matches_device_call():
    packed = inputs.workload_tensor()
    want = run_dev(packed, 4095, pm.PM_TENSOR)
    got = run_host(packed, 4095, pm.PM_TENSOR)
    assert_equal(got, want, "1024 pairs of degree 4095")
    k = np.array([0, 1, 4095, 8190])
    a, a_off, b, b_off, c_off = packed
    for i in (0, 511, 1023):
        ai, bi = a[a_off[i]:a_off[i + 1]], b[b_off[i]:b_off[i + 1]]
        ci = got[c_off[i]:c_off[i + 1]]
        assert_equal(ci[k], [oracle.coeff(ai, bi, P, int(x)) for x in k], f"pair {i} spot check")


def test_offsets_that_break_the_layout_are_refused():
    packed = inputs.workload_tensor(batch=4, deg=100, seed=inputs.SEED_BASE + 420)
    a, a_off, b, b_off, c_off = packed
    bad = np.array(c_off, np.int64)
    bad[2] += 1
    with pytest.raises(pm.PolymulError):
        run_host((a, a_off, b, b_off, bad), 100, pm.PM_PLAIN)
