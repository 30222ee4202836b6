"""The transform form's lazy modular arithmetic, emulated with 32-bit wrap-around on the CPU (no
kernel runs): Shoup's product without its final correction lands in [0, 2p) for any 32-bit input
(D. Harvey, J. Symb. Comp. 2014), Montgomery's product of inputs below 2p lands in [0, 2p)
because 4p < 2^32, and the radix-4 and radix-2 butterflies keep values in [0, 2p) while computing
the exact butterfly mod p, for primes up to 2^30 - 35."""
import numpy as np
import pytest

M32 = 0xFFFFFFFF
PRIMES = [7681, 12289, 469762049, 998244353, (1 << 30) - 35]


def umin(a, b):
    return a if a < b else b


def r2p(v, p2):
    return umin(v & M32, (v - p2) & M32)


def shoup_pair(w, p):
    return w, (w << 32) // p


def mul_shoup_lz(x, w, p):
    wv, wq = w
    return (x * wv - ((x * wq) >> 32) * p) & M32


def mul_shoup(x, w, p):
    r = mul_shoup_lz(x, w, p)
    return umin(r, (r - p) & M32)


def mul_mont_lz(x, y, p):
    pinv_neg = (-pow(p, -1, 1 << 32)) & M32
    t = x * y
    q = ((t & M32) * pinv_neg) & M32
    return (t + q * p) >> 32


def bf4t(x, w4, tws, forward, on, p):
    """The kernels' lazy radix-4 butterfly (decimation in frequency forward, in time inverse)."""
    x0, x1, x2, x3 = x
    p2 = 2 * p
    if not forward and on:
        x1, x2, x3 = (mul_shoup_lz(v, t, p) for v, t in zip((x1, x2, x3), tws))
    t0, t1 = r2p(x0 + x2, p2), r2p(x0 - x2 + p2, p2)
    t2, t3 = r2p(x1 + x3, p2), mul_shoup_lz((x1 - x3 + p2) & M32, w4, p)
    y0 = r2p(t0 + t2, p2)
    if forward and on:
        y1 = mul_shoup_lz((t1 + t3) & M32, tws[0], p)
        y2 = mul_shoup_lz((t0 - t2 + p2) & M32, tws[1], p)
        y3 = mul_shoup_lz((t1 - t3 + p2) & M32, tws[2], p)
    else:
        y1, y2, y3 = r2p(t1 + t3, p2), r2p(t0 - t2 + p2, p2), r2p(t1 - t3 + p2, p2)
    return y0, y1, y2, y3


def bf4_exact(x, w4, tw, forward, on, p):
    x0, x1, x2, x3 = x
    if not forward and on:
        x1, x2, x3 = x1 * tw[0] % p, x2 * tw[1] % p, x3 * tw[2] % p
    t0, t1, t2, t3 = (x0 + x2) % p, (x0 - x2) % p, (x1 + x3) % p, (x1 - x3) * w4 % p
    z = [(t0 + t2) % p, (t1 + t3) % p, (t0 - t2) % p, (t1 - t3) % p]
    if forward and on:
        z[1], z[2], z[3] = z[1] * tw[0] % p, z[2] * tw[1] % p, z[3] * tw[2] % p
    return z


def samples(p, rng, k=300):
    ext = [0, 1, p - 1, p, p + 1, 2 * p - 1]
    return ext + [int(v) for v in rng.integers(0, 2 * p, k)]


@pytest.mark.parametrize("p", PRIMES)
def test_shoup_and_montgomery_bounds(p):
    assert 4 * p < (1 << 32)
    rng = np.random.default_rng(p % 1000)
    ws = [0, 1, p - 1] + [int(v) for v in rng.integers(0, p, 40)]
    xs = [0, 1, M32, M32 - 1, 2 * p - 1, 4 * p - 1] + [int(v) for v in rng.integers(0, 1 << 32, 200, dtype=np.uint64)]
    for w in ws:
        wp = shoup_pair(w, p)
        for x in xs:
            r = mul_shoup_lz(x, wp, p)
            assert r < 2 * p and r % p == x * w % p
            assert mul_shoup(x, wp, p) == x * w % p
    rinv = pow(1 << 32, -1, p)
    for x in samples(p, rng, 60):
        for y in samples(p, rng, 60):
            u = mul_mont_lz(x, y, p)
            assert u < 2 * p and u % p == x * y * rinv % p


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("forward", [True, False])
def test_radix4_butterfly_stays_below_2p_and_is_exact(p, forward):
    rng = np.random.default_rng(p % 997 + forward)
    w4v = None
    # a primitive 4th root of unity mod p (p = 1 mod 4 for every prime here)
    for c in range(2, 200):
        cand = pow(c, (p - 1) // 4, p)
        if cand * cand % p == p - 1:
            w4v = cand
            break
    assert w4v is not None
    w4 = shoup_pair(w4v, p)
    vals = samples(p, rng, 40)
    for trial in range(400):
        x = [vals[int(i)] for i in rng.integers(0, len(vals), 4)]
        twv = [int(v) for v in rng.integers(0, p, 3)]
        tws = [shoup_pair(v, p) for v in twv]
        for on in (True, False):
            y = bf4t(x, w4, tws, forward, on, p)
            assert all(v < 2 * p for v in y)
            assert [v % p for v in y] == bf4_exact([v % p for v in x], w4v, twv, forward, on, p)


@pytest.mark.parametrize("p", PRIMES)
def test_radix2_butterfly_stays_below_2p_and_is_exact(p):
    rng = np.random.default_rng(p % 991)
    vals = samples(p, rng, 60)
    p2 = 2 * p
    for trial in range(600):
        u, v = (vals[int(i)] for i in rng.integers(0, len(vals), 2))
        wv = int(rng.integers(0, p))
        tv = shoup_pair(wv, p)
        # forward: (u + v, (u - v) w); inverse: (u + v w, u - v w)
        d = (u - v + p2) & M32
        fu, fv = r2p(u + v, p2), mul_shoup_lz(d, tv, p)
        assert fu < p2 and fv < p2
        assert (fu % p, fv % p) == ((u + v) % p, (u - v) * wv % p)
        w = mul_shoup_lz(v, tv, p)
        iv, iu = r2p((u - w + p2) & M32, p2), r2p(u + w, p2)
        assert iu < p2 and iv < p2
        assert (iu % p, iv % p) == ((u + v * wv) % p, (u - v * wv) % p)
