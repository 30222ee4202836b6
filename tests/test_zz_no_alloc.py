"""polymul_plain_noalloc: the allocation-free entry point, for callers that
cannot let a library call cudaMalloc (a process whose caching allocator
already holds nearly all device memory, a latency-bound caller that cannot
take the synchronisation an allocation may imply, a host whose memory policy
gives every allocation to one owner).  Its scratch lives in a static device
array.

Checked here through the C ABI: two calls in a row give exactly the words
that polymul_plain gives, which are the CPU oracle's (for several s and both
operand orders), and after
the first call (which sets the array up) the calls leave the device's free
memory unchanged.  This file is collected last so that a run stopping at the
first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1402_0264_gb300 import inputs
from paper_1402_0264_gb300 import polymul as pm
from tests.gpuhelp import assert_equal, dev, host

pytestmark = pytest.mark.gpu
P = inputs.P_DEFAULT


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_0264_gb300 import build
    build.build()


def _noalloc(lib, a, b, out, s, stream):
    return lib.polymul_plain_noalloc(ctypes.c_void_p(a.data_ptr()), a.numel() - 1,
                                     ctypes.c_void_p(b.data_ptr()), b.numel() - 1,
                                     ctypes.c_void_p(out.data_ptr()), P, s,
                                     ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_plain_on_two_calls_in_a_row():
    import torch
    lib = pm.lib()
    stream = torch.cuda.current_stream()
    # (a, b, s): the headline pair, a long a with a short b, and the operands the other way round
    cases = [(*inputs.workload_single(), 8), (*inputs.poly_pair(5000, 777, inputs.SEED_BASE + 500), 16),
             (*inputs.poly_pair(300, 9000, inputs.SEED_BASE + 501), 4),
             (*inputs.poly_pair(4097, 4097, inputs.SEED_BASE + 502), 32)]
    tensors = [(dev(a), dev(b)) for a, b, _ in cases]
    svals = [s for _, _, s in cases]
    outs = [torch.empty(a.numel() + b.numel() - 1, dtype=torch.uint32, device="cuda") for a, b in tensors]
    # the references also load every kernel instance used below and the fill kernel before
    # the free-memory baseline: lazy module loading takes device memory on first use
    refs = [host(pm.plain(a, b, s=s)) for (a, b), s in zip(tensors, svals)]
    for (a, b, s), ref in zip(cases, refs):
        assert_equal(ref, oracle.polymul(a, b, P), f"reference s={s} against the oracle")
    for out in outs:
        out.fill_(0)
    # first call on this device: sets the static array up
    assert _noalloc(lib, tensors[0][0], tensors[0][1], outs[0], svals[0], stream) == 0
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for rep in range(2):  # two calls in a row for every case; the array keeps the last call's contents
        for (a, b), out, ref, s in zip(tensors, outs, refs, svals):
            out.fill_(0)
            rc = _noalloc(lib, a, b, out, s, stream)
            assert rc == 0, pm.STATUS.get(rc, rc)
            assert_equal(host(out), ref, f"noalloc s={s}, call {rep + 1}")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before, "the calls changed the device's free memory"
    assert pm.sync_status() == 0


def test_noalloc_rejects_what_polymul_plain_rejects():
    import torch
    lib = pm.lib()
    a = dev(np.ones(10, np.uint32))
    out = torch.empty(19, dtype=torch.uint32, device="cuda")
    stream = torch.cuda.current_stream()
    assert _noalloc(lib, a, a, out, 3, stream) == 1          # s not a power of two
    assert lib.polymul_plain_noalloc(None, 9, ctypes.c_void_p(a.data_ptr()), 9,
                                     ctypes.c_void_p(out.data_ptr()), P, 8,
                                     ctypes.c_void_p(stream.cuda_stream)) == 1
