"""Python binding of libpolymul.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/polymul.h with
device pointers taken from torch CUDA tensors and the current torch stream.
There is no CPU path: tensors must live on a CUDA device and the library
must have been built (``python -m paper_1402_0264_gb300.build``); otherwise
these functions raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# POLYMUL_LIBRARY may name another build of the same ABI (the range-checked one, _build/checked/)
LIB_PATH = os.environ.get("POLYMUL_LIBRARY") or os.path.join(HERE, "_build", "libpolymul.so")

P_DEFAULT = 469762049
PM_AUTO, PM_PLAIN, PM_TENSOR = 0, 1, 2
PM_DEBUG_FAIL_ALLOC, PM_DEBUG_TC_WAIT_LIMIT = 1, 2
PM_TUNE_PLAIN, PM_TUNE_BATCHED = 1, 2
Q_CANDIDATES = (128, 256, 512, 1024, 2048)
S_CANDIDATES = (1, 2, 4, 8, 16, 32, 64)

STATUS = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_RANGE", 3: "PM_ERR_UNSUPPORTED",
          4: "PM_ERR_NOMEM", 5: "PM_ERR_CUDA", 6: "PM_ERR_TIMEOUT", 7: "PM_ERR_INTERNAL"}


class PolymulError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


_lock = threading.Lock()
_lib = None

_u32p = ctypes.c_void_p
_i64 = ctypes.c_int64


def _declare(lib):
    V, I64, U32, INT, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
    sig = {
        "polymul_plain": ([V, I64, V, I64, V, U32, INT, V], INT),
        "polymul_ntt": ([V, I64, V, I64, V, U32, U32, V], INT),
        "polymul_plain_noalloc": ([V, I64, V, I64, V, U32, INT, V], INT),
        "polymul_plain_ell": ([V, I64, V, I64, V, U32, INT, INT, V], INT),
        "polymul_batched": ([I64, V, V, V, V, V, V, U32, INT, INT, I64, V], INT),
        "polymul_batched_host": ([I64, V, V, V, V, V, V, U32, INT, INT, I64, V], INT),
        "polymul_divide": ([V, I64, V, I64, V, V, U32, INT, V], INT),
        "polymul_gcd": ([V, I64, V, I64, V, ctypes.POINTER(I64), U32, INT, V], INT),
        "polymul_model_predict": ([I64, I64, INT, INT, D, D, ctypes.POINTER(D)], INT),
        "polymul_tune_plain": ([V, I64, V, I64, V, U32, INT, V, ctypes.POINTER(INT),
                                ctypes.POINTER(ctypes.c_float)], INT),
        "polymul_plain_default_s": ([I64, I64, U32], INT),
        "polymul_sync_status": ([V], INT),
        "polymul_release": ([], INT),
        "polymul_status_string": ([INT], ctypes.c_char_p),
        "polymul_last_cuda_error": ([], INT),
        "polymul_launch_count": ([], ctypes.c_uint64),
        "polymul_debug_set": ([INT, I64], INT),
        "polymul_probe_mac_rate": ([INT, INT, I64, ctypes.POINTER(D), V], INT),
        "polymul_probe_mma": ([INT, I64, ctypes.POINTER(D), ctypes.POINTER(INT), V], INT),
        "polymul_tensor_limbs": ([ctypes.POINTER(INT), ctypes.POINTER(INT), ctypes.POINTER(U32),
                                  ctypes.POINTER(U32), ctypes.POINTER(INT), ctypes.POINTER(INT)], INT),
        "polymul_tune_batched": ([I64, V, V, V, V, V, V, U32, I64, INT, V, ctypes.POINTER(INT),
                                  ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_float)], INT),
        "polymul_tune_save": ([ctypes.c_char_p], INT),
        "polymul_tune_load": ([ctypes.c_char_p], INT),
        "polymul_tune_clear": ([], INT),
        "polymul_tune_lookup": ([ctypes.c_char_p, INT, INT, U32, I64, I64, ctypes.POINTER(INT),
                                 ctypes.POINTER(I64)], INT),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libpolymul.so not built (expected at {LIB_PATH}); run "
                                   "python -m paper_1402_0264_gb300.build")
            _lib = _declare(ctypes.CDLL(LIB_PATH))
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise PolymulError(rc, where)


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_words(t, name: str):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (no CPU path)")
    if t.element_size() != 4 or not t.is_contiguous() or t.dim() != 1:
        raise TypeError(f"{name} must be a contiguous 1-D tensor of 32-bit words")
    return ctypes.c_void_p(t.data_ptr())


def _dev_i64(t, name: str):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous int64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _alloc(n: int, like):
    torch = _torch()
    return torch.empty(n, dtype=torch.uint32, device=like.device)


def plain(a, b, p: int = P_DEFAULT, s: int = 0, out=None, stream=None):
    """c = a*b mod p by the s-blocked product (s = 0: tuned/default)."""
    L = a.numel() + b.numel() - 1
    out = _alloc(L, a) if out is None else out
    if out.numel() != L:
        raise ValueError("out must hold len(a) + len(b) - 1 words")
    _check(lib().polymul_plain(_dev_words(a, "a"), a.numel() - 1, _dev_words(b, "b"), b.numel() - 1,
                               _dev_words(out, "out"), p, s, _stream_ptr(stream)), "polymul_plain")
    return out


def plain_ell(a, b, s: int, ell: int, p: int = P_DEFAULT, out=None, stream=None):
    """plain() with l = ell threads per block (128, 256 or 512): the block-size study."""
    L = a.numel() + b.numel() - 1
    out = _alloc(L, a) if out is None else out
    if out.numel() != L:
        raise ValueError("out must hold len(a) + len(b) - 1 words")
    _check(lib().polymul_plain_ell(_dev_words(a, "a"), a.numel() - 1, _dev_words(b, "b"), b.numel() - 1,
                                   _dev_words(out, "out"), p, s, ell, _stream_ptr(stream)), "polymul_plain_ell")
    return out


def plain_noalloc(a, b, p: int = P_DEFAULT, s: int = 0, out=None, stream=None):
    """plain() with the kernel's scratch in the library's static device array (no allocation
    by the library; the caller still provides the output).  Calls must not overlap on the GPU."""
    L = a.numel() + b.numel() - 1
    out = _alloc(L, a) if out is None else out
    if out.numel() != L:
        raise ValueError("out must hold len(a) + len(b) - 1 words")
    _check(lib().polymul_plain_noalloc(_dev_words(a, "a"), a.numel() - 1, _dev_words(b, "b"),
                                       b.numel() - 1, _dev_words(out, "out"), p, s,
                                       _stream_ptr(stream)), "polymul_plain_noalloc")
    return out


def ntt(a, b, p: int = P_DEFAULT, g: int = 0, out=None, stream=None):
    """c = a*b mod p through number-theoretic transforms."""
    L = a.numel() + b.numel() - 1
    out = _alloc(L, a) if out is None else out
    if out.numel() != L:
        raise ValueError("out must hold len(a) + len(b) - 1 words")
    _check(lib().polymul_ntt(_dev_words(a, "a"), a.numel() - 1, _dev_words(b, "b"), b.numel() - 1,
                             _dev_words(out, "out"), p, g, _stream_ptr(stream)), "polymul_ntt")
    return out


def batched(a_data, a_off, b_data, b_off, c_off, max_deg: int, p: int = P_DEFAULT,
            mode: int = PM_PLAIN, s: int = 0, out=None, total: int | None = None, stream=None):
    """Products of a CSR batch; `total` = c_off[-1] (read from the device if None)."""
    batch = a_off.numel() - 1
    if total is None:
        total = int(c_off[-1].item())
    out = _alloc(total, a_data) if out is None else out
    _check(lib().polymul_batched(batch, _dev_words(a_data, "a_data"), _dev_i64(a_off, "a_off"),
                                 _dev_words(b_data, "b_data"), _dev_i64(b_off, "b_off"),
                                 _dev_words(out, "out"), _dev_i64(c_off, "c_off"), p, mode, s,
                                 max_deg, _stream_ptr(stream)), "polymul_batched")
    return out


def _host_array(t, name: str, itemsize: int):
    """(pointer, length) of a contiguous 1-D host array: a CPU tensor (pinned for overlapped
    copies) or a numpy array."""
    torch = _torch()
    if isinstance(t, torch.Tensor):
        if t.is_cuda or t.element_size() != itemsize or not t.is_contiguous() or t.dim() != 1:
            raise TypeError(f"{name} must be a contiguous 1-D CPU tensor of {8 * itemsize}-bit words")
        return ctypes.c_void_p(t.data_ptr()), t.numel()
    import numpy as np
    if not isinstance(t, np.ndarray) or t.itemsize != itemsize or t.ndim != 1 or not t.flags["C_CONTIGUOUS"]:
        raise TypeError(f"{name} must be a contiguous 1-D array of {8 * itemsize}-bit words")
    return ctypes.c_void_p(t.ctypes.data), t.size


def batched_host(a_data, a_off, b_data, b_off, c_off, out, max_deg: int, p: int = P_DEFAULT,
                 mode: int = PM_PLAIN, s: int = 0, stream=None):
    """polymul_batched_host: the products of a CSR batch whose arrays are all in host memory (CPU
    tensors or numpy arrays; pinned CPU tensors let the copies overlap the products).  `out` (host,
    c_off[-1] words) holds the products once `stream` has reached the call's end."""
    pa, na = _host_array(a_data, "a_data", 4)
    pao, nao = _host_array(a_off, "a_off", 8)
    pb, nb = _host_array(b_data, "b_data", 4)
    pbo, nbo = _host_array(b_off, "b_off", 8)
    pco, nco = _host_array(c_off, "c_off", 8)
    pc, nc = _host_array(out, "out", 4)
    batch = nao - 1
    if nbo != nao or nco != nao:
        raise ValueError("the three offset arrays must have batch + 1 entries")
    if batch > 0:
        last = [int(x[-1]) for x in (a_off, b_off, c_off)]
        if last[0] > na or last[1] > nb or last[2] > nc:
            raise ValueError("an offset array points past its data array")
    _check(lib().polymul_batched_host(batch, pa, pao, pb, pbo, pc, pco, p, mode, s, max_deg, _stream_ptr(stream)),
           "polymul_batched_host")
    return out


def divide(a, b, p: int = P_DEFAULT, s: int = 0, q=None, r=None, stream=None):
    """(q, r) with a = q b + r over Z/pZ, deg r < deg b (Section 3); s division steps per launch."""
    nq = a.numel() - b.numel() + 1
    if nq < 1:
        raise ValueError("divide needs len(a) >= len(b)")
    q = _alloc(nq, a) if q is None else q
    r = _alloc(b.numel() - 1, a) if r is None else r
    if q.numel() != nq or r.numel() != b.numel() - 1:
        raise ValueError("q must hold len(a) - len(b) + 1 words and r len(b) - 1")
    rp = _dev_words(r, "r") if r.numel() > 0 else ctypes.c_void_p(None)
    _check(lib().polymul_divide(_dev_words(a, "a"), a.numel() - 1, _dev_words(b, "b"), b.numel() - 1,
                                _dev_words(q, "q"), rp, p, s, _stream_ptr(stream)), "polymul_divide")
    return q, r


def gcd(a, b, p: int = P_DEFAULT, s: int = 0, out=None, stream=None):
    """The monic gcd of a and b over Z/pZ, p prime (Section 6); s division steps per launch.
    Returns a view of the first deg + 1 words of `out` (max(len(a), len(b)) words); synchronises
    the stream."""
    n = max(a.numel(), b.numel())
    out = _alloc(n, a) if out is None else out
    if out.numel() != n:
        raise ValueError("out must hold max(len(a), len(b)) words")
    deg = ctypes.c_int64(-2)
    _check(lib().polymul_gcd(_dev_words(a, "a"), a.numel() - 1, _dev_words(b, "b"), b.numel() - 1,
                             _dev_words(out, "out"), ctypes.byref(deg), p, s, _stream_ptr(stream)), "polymul_gcd")
    return out[: deg.value + 1]


def model_predict(n: int, m: int, s: int, ell: int, U: float, P: float) -> dict:
    """Section 5 cost formulas with Theorem 1 / Corollary 1 (host code, no GPU)."""
    out = (ctypes.c_double * 9)()
    _check(lib().polymul_model_predict(n, m, s, ell, U, P, out), "polymul_model_predict")
    keys = ("W", "S", "O", "N", "L", "C", "K", "T_thm", "T_cor")
    return dict(zip(keys, list(out)))


def tune_plain(a, b, p: int = P_DEFAULT, reps: int = 5, out=None, stream=None):
    """Times every s, records the best for this size class; returns (best_s, {s: ms})."""
    L = a.numel() + b.numel() - 1
    out = _alloc(L, a) if out is None else out
    best = ctypes.c_int(0)
    times = (ctypes.c_float * 7)()
    _check(lib().polymul_tune_plain(_dev_words(a, "a"), a.numel() - 1, _dev_words(b, "b"),
                                    b.numel() - 1, _dev_words(out, "out"), p, reps,
                                    _stream_ptr(stream), ctypes.byref(best), times),
           "polymul_tune_plain")
    return best.value, {s: t for s, t in zip(S_CANDIDATES, list(times)) if t >= 0}


def tune_batched(a_data, a_off, b_data, b_off, c_off, max_deg: int, p: int = P_DEFAULT, reps: int = 20,
                 out=None, total: int | None = None, stream=None):
    """The batched autotuner: returns (best_s, best_q, {(s, q): median ms}) and records the choice."""
    batch = a_off.numel() - 1
    if total is None:
        total = int(c_off[-1].item())
    out = _alloc(total, a_data) if out is None else out
    bs, bq = ctypes.c_int(0), ctypes.c_int64(0)
    times = (ctypes.c_float * 35)()
    _check(lib().polymul_tune_batched(batch, _dev_words(a_data, "a_data"), _dev_i64(a_off, "a_off"),
                                      _dev_words(b_data, "b_data"), _dev_i64(b_off, "b_off"),
                                      _dev_words(out, "out"), _dev_i64(c_off, "c_off"), p, max_deg, reps,
                                      _stream_ptr(stream), ctypes.byref(bs), ctypes.byref(bq), times),
           "polymul_tune_batched")
    res = {}
    for i, sv in enumerate(S_CANDIDATES):
        for j, qv in enumerate(Q_CANDIDATES):
            if times[5 * i + j] >= 0:
                res[(sv, qv)] = times[5 * i + j]
    return bs.value, bq.value, res


def tune_save(path: str):
    _check(lib().polymul_tune_save(path.encode()), "polymul_tune_save")


def tune_load(path: str):
    _check(lib().polymul_tune_load(path.encode()), "polymul_tune_load")


def tune_clear():
    _check(lib().polymul_tune_clear(), "polymul_tune_clear")


def tune_lookup(device: str, sms: int, form: int, p: int, x: int, y: int):
    """The cached (s, q) for an explicit device and size class; (0, 0) if none (host-only)."""
    s_, q_ = ctypes.c_int(0), ctypes.c_int64(0)
    _check(lib().polymul_tune_lookup(device.encode(), sms, form, p, x, y, ctypes.byref(s_), ctypes.byref(q_)),
           "polymul_tune_lookup")
    return s_.value, q_.value


def default_s(deg_a: int, deg_b: int, p: int = P_DEFAULT) -> int:
    return lib().polymul_plain_default_s(deg_a, deg_b, p)


def sync_status(stream=None) -> int:
    """Synchronises the stream; returns and clears the device status word."""
    return lib().polymul_sync_status(_stream_ptr(stream))


def launch_count() -> int:
    return int(lib().polymul_launch_count())


def probe_mac_rate(threads: int = 256, blocks_per_sm: int = 4, iters: int = 20000, stream=None) -> float:
    """32x32->64 multiply-adds per clock per SM, measured (polymul_probe_mac_rate)."""
    r = ctypes.c_double(0.0)
    _check(lib().polymul_probe_mac_rate(threads, blocks_per_sm, iters, ctypes.byref(r), _stream_ptr(stream)),
           "polymul_probe_mac_rate")
    return r.value


PM_MMA_BF16, PM_MMA_E4M3 = 0, 1


def tensor_limbs() -> dict:
    """The tensor-core form's limb encoding (polymul_tensor_limbs): limbs and bases of a and b,
    digit products per fp32 entry, tile width in blocks of 32, limb products per modular MAC."""
    na, nb, mt, tb = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    ba, bb = ctypes.c_uint32(0), ctypes.c_uint32(0)
    _check(lib().polymul_tensor_limbs(ctypes.byref(na), ctypes.byref(nb), ctypes.byref(ba), ctypes.byref(bb),
                                      ctypes.byref(mt), ctypes.byref(tb)), "polymul_tensor_limbs")
    return {"na": na.value, "nb": nb.value, "base_a": ba.value, "base_b": bb.value, "max_terms": mt.value,
            "tile_blocks": tb.value, "limb_products": na.value * nb.value}


def probe_mma(kind: int = PM_MMA_BF16, iters: int = 4096, stream=None) -> tuple[float, bool]:
    """(dense flops per clock per SM, exact fp32 accumulation) of one tcgen05 MMA kind (polymul_probe_mma)."""
    r = ctypes.c_double(0.0)
    ex = ctypes.c_int(0)
    _check(lib().polymul_probe_mma(kind, iters, ctypes.byref(r), ctypes.byref(ex), _stream_ptr(stream)),
           "polymul_probe_mma")
    return r.value, bool(ex.value)


def debug_set(knob: int, value: int):
    """Test hooks of the failure paths (polymul_debug_set)."""
    _check(lib().polymul_debug_set(knob, value), "polymul_debug_set")


def release():
    _check(lib().polymul_release(), "polymul_release")
