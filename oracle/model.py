"""Cost model of the s-blocked plain multiplication, in fp64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sources, all in Haque, Moreno Maza, Xie:
* Section 2.3: work W, span S and parallelism overhead O of a program.
* Section 2.4: Theorem 1, T_P <= (N/P + L) * C with C = max_B (S(B) + O(B)),
  and Corollary 1, T <= (N/K + L) * C with K the largest number of
  thread-blocks along an antichain of the thread-block DAG.
* Section 5 (printed, short version): for Algorithm 5 with parameter s and
  l threads per block, deg a = n-1, deg b = m-1,
      W_s = (2m - 1/2)(n + s - 1)
      S_s = 2 s^2 + s log2(m/s) - s
      O_s = (n + s - 1)(5 m s + 2 m - 3 s^2) U / (s^2 l)
      N_s = (n + s - 1)(2m - s) / (s^2 l)
      L_s = log2(m/s) + 1
      C_s = s (2s - 1) + 2 U (s + 1)
  and the local-memory constraint 2 s l + 2 s - 1 <= Z.
* Section 5, the printed ratios: W_1/W_s, S_1/S_s, O_1/O_s (m = n) and the
  Corollary-1 ratio R of the naive (s = 1) bound to the s bound.

Reading used for Corollary 1 (the paper does not spell K out for Section 5):
K is the number of MulKer thread-blocks, x*y/(s*l) with x = m/s and
y = n+s-1.  With that K, Corollary 1 applied to the formulas above gives
exactly the printed R; the tests check this.
"""
from __future__ import annotations

import math


def work(n: float, m: float, s: float) -> float:
    return (2.0 * m - 0.5) * (n + s - 1.0)


def span(n: float, m: float, s: float) -> float:
    return 2.0 * s * s + s * math.log2(m / s) - s


def overhead(n: float, m: float, s: float, ell: float, U: float) -> float:
    return (n + s - 1.0) * (5.0 * m * s + 2.0 * m - 3.0 * s * s) * U / (s * s * ell)


def blocks(n: float, m: float, s: float, ell: float) -> float:
    """N_s, the number of vertices of the thread-block DAG."""
    return (n + s - 1.0) * (2.0 * m - s) / (s * s * ell)


def levels(m: float, s: float) -> float:
    """L_s, the critical path length of the thread-block DAG."""
    return math.log2(m / s) + 1.0


def block_cost(s: float, U: float) -> float:
    """C_s = max over blocks of span + overhead."""
    return s * (2.0 * s - 1.0) + 2.0 * U * (s + 1.0)


def mulker_blocks(n: float, m: float, s: float, ell: float) -> float:
    """Thread-blocks of the one MulKer launch: x*y/(s*l), x = m/s, y = n+s-1."""
    return (m / s) * (n + s - 1.0) / (s * ell)


def local_memory_ok(s: int, ell: int, Z: int) -> bool:
    """2 s l + 2 s - 1 <= Z (words)."""
    return 2 * s * ell + 2 * s - 1 <= Z


def theorem1(n: float, m: float, s: float, ell: float, U: float, P: float) -> float:
    """Theorem 1 bound (N_s / P + L_s) * C_s, in model time units."""
    return (blocks(n, m, s, ell) / P + levels(m, s)) * block_cost(s, U)


def corollary1(n: float, m: float, s: float, ell: float, U: float) -> float:
    """Corollary 1 bound (N_s / K + L_s) * C_s with K = MulKer blocks."""
    K = mulker_blocks(n, m, s, ell)
    return (blocks(n, m, s, ell) / K + levels(m, s)) * block_cost(s, U)


# ---- the paper's printed ratios (Section 5) -------------------------------

def printed_work_ratio(n: float, s: float) -> float:
    return n / (n + s - 1.0)


def printed_span_ratio(m: float, s: float) -> float:
    return (math.log2(m) + 1.0) / (s * (math.log2(m / s) + 2.0 * s - 1.0))


def printed_overhead_ratio(n: float, s: float) -> float:
    """O_1 / O_s with m = n."""
    return n * s * s * (7.0 * n - 3.0) / ((n + s - 1.0) * (5.0 * n * s + 2.0 * n - 3.0 * s * s))


def printed_R(n: float, s: float, U: float) -> float:
    """Ratio of the Corollary-1 estimates, naive (s = 1) over s, with m = n."""
    num = (n * math.log2(n) + 3.0 * n - 1.0) * (1.0 + 4.0 * U)
    den = (n * math.log2(n / s) + 3.0 * n - s) * (2.0 * U * s + 2.0 * U + 2.0 * s * s - s)
    return num / den


def predict(n: float, m: float, s: float, ell: float, U: float, P: float) -> dict:
    """All model quantities for one (n, m, s) point."""
    return {
        "W": work(n, m, s),
        "S": span(n, m, s),
        "O": overhead(n, m, s, ell, U),
        "N": blocks(n, m, s, ell),
        "L": levels(m, s),
        "C": block_cost(s, U),
        "K": mulker_blocks(n, m, s, ell),
        "T_thm": theorem1(n, m, s, ell, U, P),
        "T_cor": corollary1(n, m, s, ell, U),
    }
