"""The matrix form of the tensor-core product, checked on the CPU with numpy (no kernel runs).

With blocks of T = 32 outputs, K running backwards (k' = 31 - k) in both operands, and for one
shift delta the M side holding the 4 limbs of b at 32 offsets r in rows (r / 8, limb j, r mod 8)
and the N side holding limb i of a's block I - delta, reversed:
    D[(j, r)][(I, i)] = sum_delta sum_{k' < 32} d_j[32 delta - 31 + r + k'] * e_i[32 (I - delta) + 31 - k']
                      = (e_i * d_j)[32 I + r],
and the M-side operand of a shift is made of 8 x 8 Hankel core matrices H_j[q] (row t, column e
= d_j[-31 + 8 q + t + e]) with q = 4 delta + r / 8 + k' / 8.  These tests build the operands by
those definitions for small random digit arrays and compare with plain convolutions."""
import numpy as np
import pytest

T = 32


def digit(arr, x):
    """arr[x] with zeros outside the array."""
    return arr[x] if 0 <= x < len(arr) else 0


def hankel(dj, q):
    return np.array([[digit(dj, -31 + 8 * q + t + e) for e in range(8)] for t in range(8)], np.int64)


def m_operand(d, delta):
    """128 x 32: row 32 g + 8 j + t (offset r = 8 g + t, limb j), column k'."""
    A = np.zeros((128, T), np.int64)
    for g in range(4):
        for j in range(len(d)):
            for t in range(8):
                r = 8 * g + t
                for kp in range(T):
                    A[32 * g + 8 * j + t, kp] = digit(d[j], T * delta - 31 + r + kp)
    return A


def n_operand(e, delta, I0, nblk):
    """(nblk * limbs) x 32: row limbs * (I - I0) + i, column k'."""
    na = len(e)
    B = np.zeros((nblk * na, T), np.int64)
    for Ir in range(nblk):
        J = I0 + Ir - delta
        for i in range(na):
            for kp in range(T):
                B[na * Ir + i, kp] = digit(e[i], T * J + 31 - kp)
    return B


@pytest.mark.parametrize("n,m,seed", [(1, 1, 0), (33, 70, 1), (200, 64, 2), (97, 150, 3)])
def test_shift_sum_is_the_digit_convolution(n, m, seed):
    rng = np.random.default_rng(seed)
    e = [rng.integers(-80, 80, n) for _ in range(4)]   # limbs of a
    d = [rng.integers(-80, 80, m) for _ in range(4)]   # limbs of b
    L = n + m - 1
    nout = (L + T - 1) // T
    nblk = 4
    for I0 in range(0, nout, nblk):
        D = np.zeros((128, nblk * 4), np.int64)
        # every shift that meets b: delta from -1 (offsets r + k' - 31 reach b[0]) to m / 32
        for delta in range(-1, (m + T - 1) // T + 1):
            D += m_operand(d, delta) @ n_operand(e, delta, I0, nblk).T
        for j in range(4):
            for i in range(4):
                conv = np.convolve(e[i], d[j])
                for Ir in range(nblk):
                    for r in range(T):
                        x = T * (I0 + Ir) + r
                        g, t = divmod(r, 8)
                        want = conv[x] if x < L else 0
                        assert D[32 * g + 8 * j + t, 4 * Ir + i] == want, (I0, Ir, r, i, j)


def test_m_operand_is_made_of_hankel_core_matrices():
    rng = np.random.default_rng(7)
    d = [rng.integers(-80, 80, 150) for _ in range(4)]
    for delta in (0, 1, 3):
        A = m_operand(d, delta)
        for g in range(4):
            for j in range(4):
                for c in range(4):
                    core = A[32 * g + 8 * j: 32 * g + 8 * j + 8, 8 * c: 8 * c + 8]
                    assert np.array_equal(core, hankel(d[j], 4 * delta + g + c))


def test_core_matrices_of_one_shift_are_reused_by_the_next():
    """Shift delta + 1 needs q = 4 delta + 4 .. 4 delta + 10: all but 4 new indices per limb are the
    ones shift delta used (q = 4 delta .. 4 delta + 6), which is what lets a slot build them once."""
    used = lambda delta: {4 * delta + g + c for g in range(4) for c in range(4)}
    for delta in range(5):
        assert len(used(delta + 1) - used(delta)) == 4
        assert used(delta) == set(range(4 * delta, 4 * delta + 7))
