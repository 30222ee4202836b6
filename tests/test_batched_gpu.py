"""Parity of the batched persistent form with the CPU oracle (every word)."""
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


def run_batch(packed, max_deg, p=P, mode=pm.PM_PLAIN, s=0):
    a_data, a_off, b_data, b_off, c_off = packed
    out = pm.batched(dev(a_data), dev64(a_off), dev(b_data), dev64(b_off), dev64(c_off),
                     max_deg=max_deg, p=p, mode=mode, s=s, total=int(c_off[-1]))
    assert pm.sync_status() == 0
    return host(out)


def test_batched_workload_full():
    """4096 pairs, degrees log-uniform in [16, 2048]."""
    packed = inputs.workload_batched()
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    assert_equal(run_batch(packed, 2048), want, "4096 pairs")


@pytest.mark.parametrize("s", [1, 2, 4, 8, 16, 32, 64])
def test_ragged_small_batch(s):
    da = np.array([0, 1, 5, 1000, 7, 0, 2047, 300, 64, 4096], np.int64)
    db = np.array([0, 3, 5, 17, 2000, 999, 2047, 1, 64, 33], np.int64)
    packed = inputs.packed_batch(da, db, 77)
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    assert_equal(run_batch(packed, 4096, s=s), want, f"s={s}")


@pytest.mark.parametrize("s", [1, 2, 4, 8, 16, 32])
def test_ragged_small_batch_warp_form(s):
    """Degrees below 4096: the warp-level form (one warp per range of positions)."""
    da = np.array([0, 1, 5, 1000, 7, 0, 2047, 300, 64, 4095, 31, 33], np.int64)
    db = np.array([0, 3, 5, 17, 2000, 999, 2047, 1, 64, 33, 4095, 32], np.int64)
    packed = inputs.packed_batch(da, db, 78)
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    assert_equal(run_batch(packed, 4095, s=s), want, f"s={s}")


@pytest.mark.parametrize("s", [4, 8])
def test_warp_form_split_tiles(s):
    """Few large pairs: every tile is cut across dozens of warps (partial-sum slots, counters)."""
    packed = inputs.packed_batch(np.array([4000, 3999, 2500], np.int64), np.array([4000, 1, 4095], np.int64), 79)
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    for rep in range(2):  # the counters are back at zero for the second call
        assert_equal(run_batch(packed, 4095, s=s), want, f"s={s} call {rep}")


def test_batch_of_one_and_unsorted_path():
    packed = inputs.packed_batch(np.array([5000]), np.array([3000]), 5)
    assert_equal(run_batch(packed, 5000), oracle.polymul_batch(*packed[:4], packed[4], P))
    # more pairs than the shared-memory sort holds: natural order path
    da = inputs.log_uniform_degrees(20000, 1, 41, 9, 1) - 1
    db = inputs.log_uniform_degrees(20000, 1, 41, 9, 2) - 1
    packed = inputs.packed_batch(da, db, 9)
    assert_equal(run_batch(packed, 40), oracle.polymul_batch(*packed[:4], packed[4], P))


def test_bad_offsets_report_invalid_arg():
    import torch
    da = np.array([10, 20, 30], np.int64)
    packed = list(inputs.packed_batch(da, da, 3))
    c_off = packed[4].copy()
    c_off[2] += 1  # pair 1 gets a wrong output length
    out = torch.full((int(c_off[-1]),), 7, dtype=torch.uint32, device="cuda")
    pm.batched(dev(packed[0]), dev64(packed[1]), dev(packed[2]), dev64(packed[3]), dev64(c_off),
               max_deg=30, out=out, total=int(c_off[-1]))
    assert pm.sync_status() == 1  # PM_ERR_INVALID_ARG from the device-side check
    assert (host(out) == 7).all()  # nothing written
    # degrees above max_deg are refused the same way
    packed = inputs.packed_batch(da, da, 3)
    pm.batched(dev(packed[0]), dev64(packed[1]), dev(packed[2]), dev64(packed[3]),
               dev64(packed[4]), max_deg=20, total=int(packed[4][-1]))
    assert pm.sync_status() == 1
    assert pm.sync_status() == 0  # cleared


def test_graph_capture_replay():
    import torch
    packed = inputs.workload_batched(batch=512)
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    a_data, a_off, b_data, b_off, c_off = [dev(x) if x.dtype == np.uint32 else dev64(x) for x in packed]
    out = torch.zeros(int(packed[4][-1]), dtype=torch.uint32, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        pm.batched(a_data, a_off, b_data, b_off, c_off, max_deg=2048, out=out, total=out.numel(), stream=st)
    st.synchronize()
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g, stream=st):
        pm.batched(a_data, a_off, b_data, b_off, c_off, max_deg=2048, out=out, total=out.numel(), stream=st)
    for _ in range(3):
        out.zero_()
        g.replay()
        assert_equal(host(out), want, "graph replay")


def test_batched_tuner_records_and_uses_its_choice(tmp_path):
    """polymul_tune_batched times (s, Q) on the warp-level schedule, records the choice for the batch's size
    class, and s = 0 calls then run with it and stay exact; the choice survives a save and a load."""
    import torch
    packed = inputs.workload_batched(batch=500)
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    t = [dev(packed[0]), dev64(packed[1]), dev(packed[2]), dev64(packed[3]), dev64(packed[4])]
    pm.tune_clear()
    best_s, best_q, times = pm.tune_batched(*t, max_deg=2048, reps=3, total=int(packed[4][-1]))
    assert best_s in (2, 4, 8, 16) and best_q in pm.Q_CANDIDATES
    assert len(times) == 20 and all(v > 0 for v in times.values())
    fastest = min(times.values())
    assert times[(best_s, best_q)] <= 1.02 * fastest + 1e-6
    props = torch.cuda.get_device_properties(0)
    key = (props.name, props.multi_processor_count, pm.PM_TUNE_BATCHED, P, 2049, 500)
    assert pm.tune_lookup(*key) == (best_s, best_q)
    assert_equal(run_batch(packed, 2048, s=0), want, "tuned s = 0 call")
    path = str(tmp_path / "tune.json")
    pm.tune_save(path)
    pm.tune_clear()
    assert pm.tune_lookup(*key) == (0, 0)
    pm.tune_load(path)
    assert pm.tune_lookup(*key) == (best_s, best_q)
    # every candidate unit size gives the same words
    for q in pm.Q_CANDIDATES:
        pm.tune_clear()
        pm.tune_load(path)
        # an entry with this Q for the same size class, then an s = 0 call
        txt = open(path).read().replace(f'"q": {best_q},', f'"q": {q},')
        open(path + ".q", "w").write(txt)
        pm.tune_load(path + ".q")
        assert pm.tune_lookup(*key) == (best_s, q)
        assert_equal(run_batch(packed, 2048, s=0), want, f"Q = {q}")
    pm.tune_clear()


@pytest.mark.parametrize("kind", ["all_small", "all_large", "mixed", "at_the_split"])
def test_auto_splits_pairs_by_size(kind):
    """PM_AUTO sends pairs whose shorter operand has at least 128 terms to the tensor cores and the
    others to the warp-level plain form, each form's planner skipping the other's pairs: batches
    with only small pairs, only large ones, both, and pairs at the boundary (127 and 128 terms) all
    match the oracle word for word."""
    rng = np.random.default_rng(1404)
    if kind == "all_small":
        da = rng.integers(0, 127, 40); db = rng.integers(0, 2000, 40)
    elif kind == "all_large":
        da = rng.integers(127, 2048, 40); db = rng.integers(127, 2048, 40)
    elif kind == "mixed":
        da = rng.integers(0, 2048, 80); db = rng.integers(0, 2048, 80)
    else:
        da = np.array([126, 127, 128, 127, 2047, 127, 0, 127]); db = np.array([127, 127, 127, 2047, 127, 126, 2047, 128])
    packed = inputs.packed_batch(da.astype(np.int64), db.astype(np.int64), 1405 + len(kind))
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    assert_equal(run_batch(packed, 2047, mode=pm.PM_AUTO), want, kind)
    assert_equal(run_batch(packed, 2047, mode=pm.PM_AUTO), want, kind + " again")
