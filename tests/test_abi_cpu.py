"""CPU checks of the C ABI: the library loads, exports every declared symbol,
validates arguments before touching the GPU, and its host cost model matches
the oracle's fp64 model.  No kernel runs here."""
import ctypes
import glob
import os
import re

import pytest

from oracle import model as omodel
from paper_1402_0264_gb300 import build as pbuild
from paper_1402_0264_gb300 import polymul as pm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return pm.lib()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(polymul_\w+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_debug_knob_validation(lib):
    assert lib.polymul_debug_set(99, 1) == 1                   # unknown knob
    assert lib.polymul_debug_set(pm.PM_DEBUG_FAIL_ALLOC, -1) == 1
    assert lib.polymul_debug_set(pm.PM_DEBUG_TC_WAIT_LIMIT, 0) == 0
    assert lib.polymul_debug_set(pm.PM_DEBUG_FAIL_ALLOC, 0) == 0


def test_probe_validation_happens_on_host(lib):
    r = ctypes.c_double(0.0)
    ex = ctypes.c_int(0)
    f = lib.polymul_probe_mma
    assert f(7, 16, ctypes.byref(r), ctypes.byref(ex), NULL) == 1           # unknown kind
    assert f(pm.PM_MMA_BF16, 0, ctypes.byref(r), ctypes.byref(ex), NULL) == 1  # no MMAs
    assert f(pm.PM_MMA_E4M3, 1 << 21, ctypes.byref(r), ctypes.byref(ex), NULL) == 1
    assert f(pm.PM_MMA_E4M3, 16, None, ctypes.byref(ex), NULL) == 1
    g = lib.polymul_probe_mac_rate
    assert g(33, 1, 100, ctypes.byref(r), NULL) == 1                         # not a multiple of 32
    assert g(256, 0, 100, ctypes.byref(r), NULL) == 1


def test_batched_host_validation_happens_on_host(lib):
    """The host-buffer batch checks its offsets and the output's overlap on the host, before any
    device work."""
    import numpy as np
    a = np.ones(8, np.uint32); b = np.ones(8, np.uint32); c = np.zeros(15, np.uint32)
    a_off = np.array([0, 8], np.int64); b_off = np.array([0, 8], np.int64); c_off = np.array([0, 15], np.int64)
    f = lib.polymul_batched_host
    ptr = lambda x: ctypes.c_void_p(x.ctypes.data)
    bad_c = np.array([0, 14], np.int64)                       # product length != n + m - 1
    assert f(1, ptr(a), ptr(a_off), ptr(b), ptr(b_off), ptr(c), ptr(bad_c), pm.P_DEFAULT, pm.PM_PLAIN, 0, 7, NULL) == 1
    assert f(1, ptr(a), ptr(a_off), ptr(b), ptr(b_off), ptr(c), ptr(c_off), pm.P_DEFAULT, pm.PM_PLAIN, 0, 6, NULL) == 1
    assert f(1, ptr(a), ptr(a_off), ptr(b), ptr(b_off), ptr(a), ptr(c_off), pm.P_DEFAULT, pm.PM_PLAIN, 0, 7, NULL) == 1
    assert f(-1, ptr(a), ptr(a_off), ptr(b), ptr(b_off), ptr(c), ptr(c_off), pm.P_DEFAULT, pm.PM_PLAIN, 0, 7, NULL) == 1
    assert f(0, ptr(a), ptr(a_off), ptr(b), ptr(b_off), ptr(c), ptr(c_off), pm.P_DEFAULT, pm.PM_PLAIN, 0, 7, NULL) == 0
    big = 1 << 25                                              # tensor form: max_deg beyond its range
    assert f(1, ptr(a), ptr(a_off), ptr(b), ptr(b_off), ptr(c), ptr(c_off), pm.P_DEFAULT, pm.PM_TENSOR, 0, big, NULL) != 0


def test_status_strings(lib):
    for code in range(8):
        assert lib.polymul_status_string(code)
    assert lib.polymul_status_string(0) == b"ok"


NULL = ctypes.c_void_p(0)
FAKE = ctypes.c_void_p(0x10000)       # never dereferenced: validation fails first
FAKE2 = ctypes.c_void_p(0x20000000)


def test_plain_validation_happens_on_host(lib):
    f = lib.polymul_plain
    assert f(NULL, 3, FAKE, 3, FAKE2, pm.P_DEFAULT, 0, NULL) == 1      # null input
    assert f(FAKE, -1, FAKE, 3, FAKE2, pm.P_DEFAULT, 0, NULL) == 1     # negative degree
    assert f(FAKE, 3, FAKE2, 2**30, FAKE2, pm.P_DEFAULT, 0, NULL) == 1  # degree too large
    assert f(FAKE, 3, FAKE2, 3, ctypes.c_void_p(0x30000000), 1, 0, NULL) == 2    # p < 2
    assert f(FAKE, 3, FAKE2, 3, ctypes.c_void_p(0x30000000), 2**30, 0, NULL) == 2  # p too large
    assert f(FAKE, 3, FAKE2, 3, ctypes.c_void_p(0x30000000), 7, 3, NULL) == 1    # s not a power of two
    assert f(FAKE, 3, FAKE2, 3, ctypes.c_void_p(0x30000000), 7, 128, NULL) == 1  # s too large
    # c overlapping a: [0x10000, +7 words) vs [0x10008, ...)
    assert f(FAKE, 3, FAKE2, 3, ctypes.c_void_p(0x10008), 7, 0, NULL) == 1


def test_batched_validation_happens_on_host(lib):
    f = lib.polymul_batched
    assert f(0, NULL, NULL, NULL, NULL, NULL, NULL, 7, 1, 0, 10, NULL) == 0   # empty batch: no-op
    assert f(-1, FAKE, FAKE, FAKE, FAKE, FAKE2, FAKE, 7, 1, 0, 10, NULL) == 1
    assert f(4, FAKE, NULL, FAKE, FAKE, FAKE2, FAKE, 7, 1, 0, 10, NULL) == 1
    assert f(4, FAKE, FAKE, FAKE, FAKE, FAKE2, FAKE, 7, 9, 0, 10, NULL) == 1  # bad mode
    assert f(4, FAKE, FAKE, FAKE, FAKE, FAKE2, FAKE, 7, 1, 5, 10, NULL) == 1  # bad s
    assert f(4, FAKE, FAKE, FAKE, FAKE, FAKE2, FAKE, 1, 1, 0, 10, NULL) == 2  # bad p
    assert f(4, FAKE, FAKE, FAKE, FAKE, FAKE2, FAKE, 7, 1, 0, -1, NULL) == 1  # bad max_deg
    # tensor mode outside its exactness bounds
    assert f(4, FAKE, FAKE, FAKE, FAKE, FAKE2, FAKE, 2**29 + 11, 2, 0, 100, NULL) == 3
    assert f(4, FAKE, FAKE, FAKE, FAKE, FAKE2, FAKE, 7, 2, 0, 2**24, NULL) == 3


def test_ntt_validation_happens_on_host(lib):
    f = lib.polymul_ntt
    assert f(NULL, 3, FAKE, 3, FAKE2, pm.P_DEFAULT, 0, NULL) == 1
    assert f(FAKE, 3, FAKE2, 3, ctypes.c_void_p(0x30000000), 2**30 + 1, 0, NULL) == 2


@pytest.mark.parametrize("n,m", [(4000, 4000), (8000, 1000), (16384, 16384), (1024, 1024)])
@pytest.mark.parametrize("s", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("U", [1.5, 22.0, 400.0])
def test_model_matches_oracle(lib, n, m, s, U):
    got = pm.model_predict(n, m, s, 256, U, 152.0)
    want = omodel.predict(n, m, s, 256, U, 152.0)
    for k, v in want.items():
        assert abs(got[k] - v) <= 1e-12 * abs(v), k


def test_model_rejects_bad_args(lib):
    with pytest.raises(pm.PolymulError):
        pm.model_predict(100, 4, 8, 256, 10.0, 152.0)   # s > m
    with pytest.raises(pm.PolymulError):
        pm.model_predict(100, 100, 4, 256, 0.0, 152.0)  # U <= 0


def test_divide_validation_happens_on_host(lib):
    f = lib.polymul_divide
    Q = ctypes.c_void_p(0x30000000)
    R = ctypes.c_void_p(0x40000000)
    P = pm.P_DEFAULT
    assert f(NULL, 5, FAKE2, 3, Q, R, P, 0, NULL) == 1          # null dividend
    assert f(FAKE, 5, FAKE2, 3, Q, NULL, P, 0, NULL) == 1       # null remainder with deg b > 0
    assert f(FAKE, 2, FAKE2, 3, Q, R, P, 0, NULL) == 1          # deg a < deg b
    assert f(FAKE, 5, FAKE2, -1, Q, R, P, 0, NULL) == 1         # negative degree
    assert f(FAKE, 5, FAKE2, 3, Q, R, 1, 0, NULL) == 2          # p < 2
    assert f(FAKE, 5, FAKE2, 3, Q, R, P, 257, NULL) == 1        # s too large
    assert f(FAKE, 5, FAKE2, 3, Q, R, P, -1, NULL) == 1         # negative s
    assert f(FAKE, 5, FAKE2, 3, FAKE, R, P, 0, NULL) == 1       # q overlapping a
    assert f(FAKE, 5, FAKE2, 3, Q, Q, P, 0, NULL) == 1          # r overlapping q


def test_plain_ell_validation_happens_on_host(lib):
    f = lib.polymul_plain_ell
    C = ctypes.c_void_p(0x30000000)
    P = pm.P_DEFAULT
    assert f(FAKE, 3, FAKE2, 3, C, P, 8, 200, NULL) == 1     # l not 128/256/512
    assert f(FAKE, 3, FAKE2, 3, C, P, 0, 256, NULL) == 1     # s must be given
    assert f(FAKE, 3, FAKE2, 3, C, P, 3, 128, NULL) == 1     # s not a power of two
    assert f(NULL, 3, FAKE2, 3, C, P, 8, 512, NULL) == 1     # null input


def test_gcd_validation_happens_on_host(lib):
    f = lib.polymul_gcd
    G = ctypes.c_void_p(0x30000000)
    P = pm.P_DEFAULT
    deg = ctypes.c_int64(0)
    dp = ctypes.byref(deg)
    assert f(NULL, 5, FAKE2, 3, G, dp, P, 0, NULL) == 1         # null input
    assert f(FAKE, 5, FAKE2, 3, G, None, P, 0, NULL) == 1       # null degree output
    assert f(FAKE, -1, FAKE2, 3, G, dp, P, 0, NULL) == 1        # negative degree
    assert f(FAKE, 5, FAKE2, 2**30, G, dp, P, 0, NULL) == 1     # degree too large
    assert f(FAKE, 5, FAKE2, 3, G, dp, 1, 0, NULL) == 2         # p < 2
    assert f(FAKE, 5, FAKE2, 3, G, dp, 2**30, 0, NULL) == 2     # p too large
    assert f(FAKE, 5, FAKE2, 3, G, dp, P, 257, NULL) == 1       # s too large
    assert f(FAKE, 5, FAKE2, 3, G, dp, P, -1, NULL) == 1        # negative s
    assert f(FAKE, 5, FAKE2, 3, FAKE, dp, P, 0, NULL) == 1      # g overlapping a
    assert f(FAKE, 5, FAKE2, 3, FAKE2, dp, P, 0, NULL) == 1     # g overlapping b


def test_binding_refuses_host_tensors(lib):
    """The product path has no CPU fallback: every entry point of the binding refuses host tensors
    before anything reaches the library."""
    import torch
    a = torch.ones(16, dtype=torch.uint32)
    b = torch.ones(9, dtype=torch.uint32)
    off = torch.tensor([0, 16], dtype=torch.int64)
    calls = [
        lambda: pm.plain(a, b),
        lambda: pm.plain_ell(a, b, 8, 128),
        lambda: pm.plain_noalloc(a, b),
        lambda: pm.ntt(a, b),
        lambda: pm.divide(a, b),
        lambda: pm.gcd(a, b),
        lambda: pm.batched(a, off, a, off, torch.tensor([0, 31], dtype=torch.int64), max_deg=15),
    ]
    for call in calls:
        with pytest.raises(TypeError):
            call()
