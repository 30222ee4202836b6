"""The transform form's algebra, checked on the CPU with Python integers (no kernel runs):
the radix-4 (and one radix-2) decimation-in-frequency network leaves the transform in the order
the frequency map gives, the decimation-in-time inverse undoes it (times the length), the
bit-reversal form of the frequency map equals the digit form, and the four-step decomposition
N = N1 N2 reproduces the length-N transform."""
import numpy as np
import pytest

P = 469762049   # 7 * 2^26 + 1, generator 3
G = 3


def root(M, inverse=False):
    w = pow(G, (P - 1) // M, P)
    return pow(w, P - 2, P) if inverse else w


def dft(x, M, inverse=False):
    w = root(M, inverse)
    return [sum(x[n] * pow(w, n * k % M, P) for n in range(M)) % P for k in range(M)]


def freq_of_pos(pos, logm):
    """Base-4 digits of the position read in reverse, after the leading binary digit when logm is
    odd (which becomes the lowest digit of the frequency)."""
    k, mult, lg, rem = 0, 1, logm, pos
    if lg & 1:
        lg -= 1
        k += (rem >> lg) * mult
        rem &= (1 << lg) - 1
        mult <<= 1
    while lg > 0:
        lg -= 2
        k += (rem >> lg) * mult
        rem &= (1 << lg) - 1
        mult <<= 2
    return k


def freq_of_pos_fast(pos, logm):
    """The same map through a bit reversal followed by a swap of the bits of every pair."""
    lg, hi, rest = logm, 0, pos
    if lg & 1:
        lg -= 1
        hi = rest >> lg
        rest &= (1 << lg) - 1
    if lg == 0:
        return hi
    r = int(format(rest, f"0{lg}b")[::-1], 2)
    r = ((r & 0x55555555) << 1) | ((r >> 1) & 0x55555555)
    return hi + 2 * r if logm & 1 else r


def network(x, logm, forward):
    """The in-place network: forward = radix-2 stage of span M/2 (odd logm) then radix-4 levels of
    span M/4^.. down to 1, twiddles on the outputs; inverse = the same levels in reverse order with
    inverse twiddles on the inputs, the radix-2 stage last."""
    M = 1 << logm
    x = list(x)
    w = root(M, inverse=not forward)
    tw = [pow(w, e, P) for e in range(M)]
    w4 = tw[M >> 2] if M >= 4 else 1
    if forward and logm & 1:
        h = M >> 1
        for j in range(h):
            u, v = x[j], x[j + h]
            x[j], x[j + h] = (u + v) % P, (u - v) * tw[j] % P
    smax = (M >> 3) if logm & 1 else (M >> 2)
    spans = []
    s = smax
    while s >= 1:
        spans.append(s)
        s >>= 2
    if not forward:
        spans.reverse()
    for s in spans:
        lgs = s.bit_length() - 1
        lgstep = logm - 2 - lgs
        for b in range(M >> 2):
            blk, j = b >> lgs, b & (s - 1)
            o = (blk << (lgs + 2)) + j
            e = j << lgstep
            x0, x1, x2, x3 = x[o], x[o + s], x[o + 2 * s], x[o + 3 * s]
            if not forward:
                x1, x2, x3 = x1 * tw[e] % P, x2 * tw[2 * e] % P, x3 * tw[3 * e] % P
            t0, t1 = (x0 + x2) % P, (x0 - x2) % P
            t2, t3 = (x1 + x3) % P, (x1 - x3) * w4 % P
            z0, z2, z1, z3 = (t0 + t2) % P, (t0 - t2) % P, (t1 + t3) % P, (t1 - t3) % P
            if forward:
                z1, z2, z3 = z1 * tw[e] % P, z2 * tw[2 * e] % P, z3 * tw[3 * e] % P
            x[o], x[o + s], x[o + 2 * s], x[o + 3 * s] = z0, z1, z2, z3
    if not forward and logm & 1:
        h = M >> 1
        for j in range(h):
            u, v = x[j], x[j + h] * tw[j] % P
            x[j], x[j + h] = (u + v) % P, (u - v) % P
    return x


@pytest.mark.parametrize("logm", range(1, 10))
def test_forward_network_order_and_inverse(logm):
    M = 1 << logm
    rng = np.random.default_rng(100 + logm)
    x = [int(v) for v in rng.integers(0, P, M)]
    X = dft(x, M)
    y = network(x, logm, forward=True)
    for pos in range(M):
        assert y[pos] == X[freq_of_pos(pos, logm)], (logm, pos)
    z = network(y, logm, forward=False)
    assert z == [M * v % P for v in x]


@pytest.mark.parametrize("logm", range(0, 25))
def test_fast_frequency_map_equals_digit_form(logm):
    M = 1 << logm
    positions = range(M) if M <= 4096 else np.random.default_rng(logm).integers(0, M, 4096)
    for pos in positions:
        assert freq_of_pos_fast(int(pos), logm) == freq_of_pos(int(pos), logm)
    if M <= 4096:  # a permutation
        assert sorted(freq_of_pos(p, logm) for p in range(M)) == list(range(M))


@pytest.mark.parametrize("N1,N2", [(2, 16), (4, 16), (8, 8), (16, 4)])
def test_four_step_decomposition(N1, N2):
    """X[k1 + N1 k2] = sum_n2 w_N2^(n2 k2) w_N^(n2 k1) sum_n1 x[n1 N2 + n2] w_N1^(n1 k1)."""
    N = N1 * N2
    rng = np.random.default_rng(N1 * 100 + N2)
    x = [int(v) for v in rng.integers(0, P, N)]
    X = dft(x, N)
    wN, w1, w2 = root(N), root(N1), root(N2)
    for k1 in range(N1):
        col = [sum(x[n1 * N2 + n2] * pow(w1, n1 * k1, P) for n1 in range(N1)) * pow(wN, n2 * k1, P) % P
               for n2 in range(N2)]
        for k2 in range(N2):
            assert X[k1 + N1 * k2] == sum(col[n2] * pow(w2, n2 * k2, P) for n2 in range(N2)) % P
