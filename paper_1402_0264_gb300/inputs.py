"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds no polynomial arithmetic: it only turns a seed into
coefficient arrays and degree lists.  Both the CUDA path and the CPU oracle
are fed from here, so neither needs the other to build its inputs.

Generator: splitmix64 used as a counter-based stream (value i of stream
(seed, stream_id) is mix(seed + stream_id * 2^32 + i + 1)), following
Steele, Lea and Flood, "Fast splittable pseudorandom number generators"
(OOPSLA 2014).  A 64-bit draw u is mapped into [0, p) by floor(u * p / 2^64),
Lemire's multiply-shift range reduction.  Everything is vectorised numpy
uint64 arithmetic, so the arrays are identical on x86_64 and aarch64.

The paper's Table 1 uses dense random polynomials with unspecified
coefficient distributions; these generators stand in for them with uniform
residues, as the workloads here specify.
"""
from __future__ import annotations

import math

import numpy as np

P_DEFAULT = 469762049  # 7 * 2^26 + 1
SEED_BASE = 0x14020264

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK32 = np.uint64(0xFFFFFFFF)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Draws `count` 64-bit values of stream (seed, stream), starting at index `start`."""
    with np.errstate(over="ignore"):
        base = np.uint64((seed + (stream << 32)) & 0xFFFFFFFFFFFFFFFF)
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(base + idx * _GOLDEN)


def uniform_mod(seed: int, stream: int, count: int, p: int = P_DEFAULT) -> np.ndarray:
    """`count` uint32 values uniform in [0, p) (p < 2^32)."""
    if not (2 <= p < 2**32):
        raise ValueError("p must be in [2, 2^32)")
    u = splitmix64(seed, stream, count)
    hi = u >> np.uint64(32)
    lo = u & _MASK32
    pp = np.uint64(p)
    with np.errstate(over="ignore"):
        # floor(u * p / 2^64) = floor((hi*p + floor(lo*p / 2^32)) / 2^32); no term overflows.
        t = hi * pp + ((lo * pp) >> np.uint64(32))
    return (t >> np.uint64(32)).astype(np.uint32)


def uniform_unit(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` float64 values in [0, 1) from the top 53 bits of each draw."""
    u = splitmix64(seed, stream, count)
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def poly_pair(deg_a: int, deg_b: int, seed: int, p: int = P_DEFAULT):
    """A pair (a, b) of dense polynomials with uniform coefficients in [0, p)."""
    a = uniform_mod(seed, 1, deg_a + 1, p)
    b = uniform_mod(seed, 2, deg_b + 1, p)
    return a, b


def log_uniform_degrees(count: int, lo: int, hi: int, seed: int, stream: int) -> np.ndarray:
    """Degrees floor(exp(U[ln lo, ln(hi+1)))) clamped to [lo, hi] (int64)."""
    u = uniform_unit(seed, stream, count)
    x = np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))
    return np.clip(np.floor(x).astype(np.int64), lo, hi)


def packed_batch(degs_a: np.ndarray, degs_b: np.ndarray, seed: int, p: int = P_DEFAULT):
    """Packs a batch of pairs into CSR form.

    Returns (a_data, a_off, b_data, b_off, c_off) where pair i occupies
    a_data[a_off[i]:a_off[i+1]] (deg_a[i]+1 words), likewise for b, and its
    product occupies c_off[i]:c_off[i+1] (deg_a[i]+deg_b[i]+1 words).
    """
    na = np.asarray(degs_a, dtype=np.int64) + 1
    nb = np.asarray(degs_b, dtype=np.int64) + 1
    a_off = np.zeros(len(na) + 1, dtype=np.int64)
    b_off = np.zeros(len(nb) + 1, dtype=np.int64)
    c_off = np.zeros(len(na) + 1, dtype=np.int64)
    np.cumsum(na, out=a_off[1:])
    np.cumsum(nb, out=b_off[1:])
    np.cumsum(na + nb - 1, out=c_off[1:])
    a_data = uniform_mod(seed, 1, int(a_off[-1]), p)
    b_data = uniform_mod(seed, 2, int(b_off[-1]), p)
    return a_data, a_off, b_data, b_off, c_off


# ---------------------------------------------------------------------------
# The five synthetic workloads (sizes, seeds and shapes in one place).
# ---------------------------------------------------------------------------

def workload_small(p: int = P_DEFAULT):
    """One pair, both of degree 1023 (seed SEED_BASE + 0)."""
    return poly_pair(1023, 1023, SEED_BASE + 0, p)


def workload_single(p: int = P_DEFAULT):
    """One pair, both of degree 16383 (seed SEED_BASE + 1)."""
    return poly_pair(16383, 16383, SEED_BASE + 1, p)


def workload_batched_degrees(batch: int = 4096, seed: int = SEED_BASE + 2):
    """Degrees log-uniform in [16, 2048], drawn independently per operand."""
    da = log_uniform_degrees(batch, 16, 2048, seed, 11)
    db = log_uniform_degrees(batch, 16, 2048, seed, 12)
    return da, db


def workload_batched(batch: int = 4096, p: int = P_DEFAULT, seed: int = SEED_BASE + 2):
    da, db = workload_batched_degrees(batch, seed)
    return packed_batch(da, db, seed, p)


def workload_tensor(batch: int = 1024, deg: int = 4095, p: int = P_DEFAULT,
                    seed: int = SEED_BASE + 3):
    """`batch` pairs of equal degree `deg` (1024 pairs of degree 4095 by default)."""
    d = np.full(batch, deg, dtype=np.int64)
    return packed_batch(d, d, seed, p)


def workload_ntt(deg: int = 2**22 - 1, p: int = P_DEFAULT, seed: int = SEED_BASE + 4):
    """One pair of degree `deg` (2^22 - 1 by default)."""
    return poly_pair(deg, deg, seed, p)


def gcd_factors(deg_g: int, deg_u: int, deg_w: int, seed: int, p: int = P_DEFAULT):
    """Factors of a planted gcd: g monic of degree deg_g and u, w uniform with nonzero leading
    coefficients.  The gcd workload is b = g u and a = g (u w + 1), whose gcd is exactly g
    (gcd(u w + 1, u) = 1); each side forms those products with its own code."""
    g = uniform_mod(seed, 21, deg_g + 1, p)
    g[-1] = 1
    u = uniform_mod(seed, 22, deg_u + 1, p)
    w = uniform_mod(seed, 23, deg_w + 1, p)
    u[-1] = u[-1] if u[-1] else 1
    w[-1] = w[-1] if w[-1] else 1
    return g, u, w


def gcd_cofactors(deg_g: int, deg_u: int, deg_v: int, seed: int, p: int = P_DEFAULT):
    """g monic of degree deg_g and independent uniform u, v with nonzero leading coefficients:
    a = g u and b = g v have gcd g whenever gcd(u, v) = 1 (true for all but a fraction of about
    1/p of draws; a test checks it for the seeds used here).  Unlike gcd_factors, the Euclidean
    algorithm on (a, b) then runs the normal remainder sequence, one degree at a time."""
    g = uniform_mod(seed, 31, deg_g + 1, p)
    g[-1] = 1
    u = uniform_mod(seed, 32, deg_u + 1, p)
    v = uniform_mod(seed, 33, deg_v + 1, p)
    u[-1] = u[-1] if u[-1] else 1
    v[-1] = v[-1] if v[-1] else 1
    return g, u, v


def workload_gcd(p: int = P_DEFAULT, seed: int = SEED_BASE + 7):
    """Factors for a of degree 9999 and b of degree 8999 with a gcd of degree 1000 (the largest
    size of the paper's gcd timings, Section 6): a = g u, b = g v with deg u = 8999, deg v = 7999."""
    return gcd_cofactors(1000, 8999, 7999, seed, p)
