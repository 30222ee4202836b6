"""CPU oracle for the polynomial-multiplication hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library in
``paper_1402_0264_gb300`` never imports it and shares no code with it.

* ``polymul``/``coeff``/``evaluate``/``ntt_polymul``: thin ctypes wrappers over
  ``polymul_oracle.c`` (the long-multiplication definition of Section 5 of
  Haque, Moreno Maza, Xie, and a textbook radix-2 NTT used only as a faster
  exact evaluator).
* ``divide``/``invmod``: Euclidean division a = q b + r over Z/pZ (Section 3),
  one division step at a time from the top as in Algorithm 1.
* ``gcd``: the monic greatest common divisor over Z/pZ (Section 6), by the
  textbook remainder sequence.
* ``polymul_omp``/``polymul_batch_omp``: the same definition shared out over
  all host threads with OpenMP (``polymul_oracle_omp.c``), for timing the CPU
  baseline only; pinned to the single-thread functions.
* ``model``: the printed cost formulas of Section 5 and the Graham-Brent bound
  of Section 2.4 (Theorem 1, Corollary 1), in fp64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polymul_oracle.c")
_SRC_OMP = os.path.join(_HERE, "polymul_oracle_omp.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libpolymul_oracle.so")
_lock = threading.Lock()
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compiles the C oracle with gcc (plain -O2, no target-specific flags).  The multi-core
    timing variants of polymul_oracle_omp.c use OpenMP where gcc has it, else one thread."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_OMP))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, _SRC_OMP]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_polymul.argtypes = [_u32p, ctypes.c_int64, _u32p, ctypes.c_int64,
                                           ctypes.c_uint32, _u32p]
            lib.oracle_polymul.restype = ctypes.c_int
            lib.oracle_coeff.argtypes = [_u32p, ctypes.c_int64, _u32p, ctypes.c_int64,
                                         ctypes.c_uint32, ctypes.c_int64]
            lib.oracle_coeff.restype = ctypes.c_uint32
            lib.oracle_eval.argtypes = [_u32p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_eval.restype = ctypes.c_uint32
            lib.oracle_powmod.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
            lib.oracle_powmod.restype = ctypes.c_uint32
            lib.oracle_ntt_polymul.argtypes = [_u32p, ctypes.c_int64, _u32p, ctypes.c_int64,
                                               ctypes.c_uint32, ctypes.c_uint32, _u32p]
            lib.oracle_ntt_polymul.restype = ctypes.c_int
            for name in ("oracle_polymul_batch",):
                fn = getattr(lib, name)
                fn.argtypes = [ctypes.c_int64, _u32p, _i64p, _u32p, _i64p, _u32p, _i64p,
                               ctypes.c_uint32]
                fn.restype = ctypes.c_int
            lib.oracle_ntt_polymul_batch.argtypes = [ctypes.c_int64, _u32p, _i64p, _u32p, _i64p,
                                                     _u32p, _i64p, ctypes.c_uint32,
                                                     ctypes.c_uint32]
            lib.oracle_ntt_polymul_batch.restype = ctypes.c_int
            lib.oracle_invmod.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_invmod.restype = ctypes.c_uint32
            lib.oracle_divide.argtypes = [_u32p, ctypes.c_int64, _u32p, ctypes.c_int64, ctypes.c_uint32,
                                          _u32p, _u32p]
            lib.oracle_divide.restype = ctypes.c_int
            lib.oracle_gcd.argtypes = [_u32p, ctypes.c_int64, _u32p, ctypes.c_int64, ctypes.c_uint32,
                                       _u32p, _i64p]
            lib.oracle_gcd.restype = ctypes.c_int
            lib.oracle_omp_threads.argtypes = []
            lib.oracle_omp_threads.restype = ctypes.c_int
            lib.oracle_polymul_omp.argtypes = [_u32p, ctypes.c_int64, _u32p, ctypes.c_int64,
                                               ctypes.c_uint32, _u32p]
            lib.oracle_polymul_omp.restype = ctypes.c_int
            lib.oracle_polymul_batch_omp.argtypes = [ctypes.c_int64, _u32p, _i64p, _u32p, _i64p, _u32p,
                                                     _i64p, ctypes.c_uint32]
            lib.oracle_polymul_batch_omp.restype = ctypes.c_int
            _lib = lib
    return _lib


def _u32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint32))


def _i64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.int64))


def _p(arr: np.ndarray, t):
    return arr.ctypes.data_as(t)


def polymul(a, b, p: int) -> np.ndarray:
    """f = a*b mod p by the long-multiplication definition (Section 5)."""
    a, b = _u32(a), _u32(b)
    f = np.zeros(len(a) + len(b) - 1, dtype=np.uint32)
    rc = _load().oracle_polymul(_p(a, _u32p), len(a), _p(b, _u32p), len(b), p, _p(f, _u32p))
    if rc != 0:
        raise ValueError("oracle_polymul: bad sizes")
    return f


def coeff(a, b, p: int, k: int) -> int:
    """One coefficient f[k] of a*b mod p, by the definition."""
    a, b = _u32(a), _u32(b)
    return int(_load().oracle_coeff(_p(a, _u32p), len(a), _p(b, _u32p), len(b), p, k))


def evaluate(poly, p: int, x: int) -> int:
    """poly(x) mod p by Horner's rule."""
    poly = _u32(poly)
    return int(_load().oracle_eval(_p(poly, _u32p), len(poly), p, x))


def powmod(base: int, e: int, p: int) -> int:
    return int(_load().oracle_powmod(base, e, p))


def ntt_polymul(a, b, p: int, g: int = 3) -> np.ndarray:
    """a*b mod p through a textbook radix-2 NTT (exact; needs 2^k | p-1)."""
    a, b = _u32(a), _u32(b)
    f = np.zeros(len(a) + len(b) - 1, dtype=np.uint32)
    rc = _load().oracle_ntt_polymul(_p(a, _u32p), len(a), _p(b, _u32p), len(b), p, g,
                                    _p(f, _u32p))
    if rc != 0:
        raise ValueError(f"oracle_ntt_polymul failed ({rc})")
    return f


def polymul_batch(a_data, a_off, b_data, b_off, c_off, p: int) -> np.ndarray:
    a_data, b_data = _u32(a_data), _u32(b_data)
    a_off, b_off, c_off = _i64(a_off), _i64(b_off), _i64(c_off)
    f = np.zeros(int(c_off[-1]), dtype=np.uint32)
    rc = _load().oracle_polymul_batch(len(a_off) - 1, _p(a_data, _u32p), _p(a_off, _i64p),
                                      _p(b_data, _u32p), _p(b_off, _i64p), _p(f, _u32p),
                                      _p(c_off, _i64p), p)
    if rc != 0:
        raise ValueError("oracle_polymul_batch: bad sizes")
    return f


def ntt_polymul_batch(a_data, a_off, b_data, b_off, c_off, p: int, g: int = 3) -> np.ndarray:
    a_data, b_data = _u32(a_data), _u32(b_data)
    a_off, b_off, c_off = _i64(a_off), _i64(b_off), _i64(c_off)
    f = np.zeros(int(c_off[-1]), dtype=np.uint32)
    rc = _load().oracle_ntt_polymul_batch(len(a_off) - 1, _p(a_data, _u32p), _p(a_off, _i64p),
                                          _p(b_data, _u32p), _p(b_off, _i64p), _p(f, _u32p),
                                          _p(c_off, _i64p), p, g)
    if rc != 0:
        raise ValueError(f"oracle_ntt_polymul_batch failed ({rc})")
    return f


def omp_threads() -> int:
    """Threads the multi-core timing variants use."""
    return int(_load().oracle_omp_threads())


def polymul_omp(a, b, p: int) -> np.ndarray:
    """polymul() with its coefficients shared out over all host threads (timing only)."""
    a, b = _u32(a), _u32(b)
    f = np.zeros(len(a) + len(b) - 1, dtype=np.uint32)
    rc = _load().oracle_polymul_omp(_p(a, _u32p), len(a), _p(b, _u32p), len(b), p, _p(f, _u32p))
    if rc != 0:
        raise ValueError("oracle_polymul_omp: bad sizes")
    return f


def polymul_batch_omp(a_data, a_off, b_data, b_off, c_off, p: int) -> np.ndarray:
    """polymul_batch() with the pairs shared out over all host threads (timing only)."""
    a_data, b_data = _u32(a_data), _u32(b_data)
    a_off, b_off, c_off = _i64(a_off), _i64(b_off), _i64(c_off)
    f = np.zeros(int(c_off[-1]), dtype=np.uint32)
    rc = _load().oracle_polymul_batch_omp(len(a_off) - 1, _p(a_data, _u32p), _p(a_off, _i64p),
                                          _p(b_data, _u32p), _p(b_off, _i64p), _p(f, _u32p),
                                          _p(c_off, _i64p), p)
    if rc != 0:
        raise ValueError("oracle_polymul_batch_omp: bad sizes")
    return f


def invmod(x: int, p: int) -> int:
    """x^-1 mod p (0 when x has no inverse)."""
    return int(_load().oracle_invmod(x, p))


def divide(a, b, p: int):
    """(q, r) with a = q b + r over Z/pZ and deg r < deg b (Section 3); len(a) >= len(b) >= 1,
    b's leading coefficient invertible mod p.  q has len(a)-len(b)+1 words, r has len(b)-1."""
    a, b = _u32(a), _u32(b)
    q = np.zeros(len(a) - len(b) + 1 if len(a) >= len(b) else 0, dtype=np.uint32)
    r = np.zeros(max(len(b) - 1, 0), dtype=np.uint32)
    rc = _load().oracle_divide(_p(a, _u32p), len(a), _p(b, _u32p), len(b), p, _p(q, _u32p),
                               _p(r, _u32p))
    if rc == -1:
        raise ValueError("oracle_divide: needs len(a) >= len(b) >= 1")
    if rc == -2:
        raise ValueError("oracle_divide: the leading coefficient of b has no inverse mod p")
    if rc != 0:
        raise MemoryError("oracle_divide")
    return q, r


def gcd(a, b, p: int):
    """The monic gcd of a and b over Z/pZ, p prime (Section 6), as a uint32 array of deg + 1
    words; an empty array when a = b = 0.  Leading zero coefficients are allowed."""
    a, b = _u32(a), _u32(b)
    g = np.zeros(max(len(a), len(b), 1), dtype=np.uint32)
    deg = ctypes.c_int64(-1)
    rc = _load().oracle_gcd(_p(a, _u32p), len(a), _p(b, _u32p), len(b), p, _p(g, _u32p),
                            ctypes.byref(deg))
    if rc == -2:
        raise ValueError("oracle_gcd: a leading coefficient has no inverse mod p")
    if rc != 0:
        raise MemoryError("oracle_gcd")
    return g[: deg.value + 1].copy()
