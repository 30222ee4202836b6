"""Independent exact references used to pin the oracle (never the CUDA path).

* kronecker_product: the exact integer convolution through one big-integer
  multiplication (Kronecker substitution), then reduction mod p.  Python's
  integer multiply is the library routine; no loop over coefficient pairs.
* horner: polynomial evaluation in Python integers.
"""
from __future__ import annotations

import numpy as np

_CHUNK = 12  # bytes per packed coefficient: sums of up to 2^31 products of 32-bit words fit


def _pack(x: np.ndarray) -> int:
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint32))
    buf = np.zeros((len(x), _CHUNK), dtype=np.uint8)
    buf[:, :4] = x.astype("<u4").view(np.uint8).reshape(len(x), 4)
    return int.from_bytes(buf.tobytes(), "little")


def kronecker_product(a, b, p: int) -> np.ndarray:
    """Exact (a*b) mod p via a(2^96) * b(2^96) in Python big integers."""
    a = np.asarray(a, dtype=np.uint32)
    b = np.asarray(b, dtype=np.uint32)
    L = len(a) + len(b) - 1
    prod = _pack(a) * _pack(b)
    raw = prod.to_bytes(L * _CHUNK, "little")
    out = np.empty(L, dtype=np.uint32)
    for k in range(L):
        v = int.from_bytes(raw[k * _CHUNK:(k + 1) * _CHUNK], "little")
        out[k] = v % p
    return out


def horner(poly, x: int, p: int) -> int:
    acc = 0
    for c in reversed([int(v) for v in poly]):
        acc = (acc * x + c) % p
    return acc
