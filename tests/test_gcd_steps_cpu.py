"""The step rule of the GPU gcd, checked on the CPU against the paper's and the oracle's (no kernel
runs).  Section 6 reduces the polynomial of larger degree (a when the degrees are equal) by
r <- r - lc(r) lc(d)^-1 x^(deg r - deg d) d.  The kernels take the fraction-free step
r <- lc(d) r - lc(r) x^(deg r - deg d) d instead, optionally times the unit 2^-32 (Montgomery's
reduction without conversion), and stop on a zero polynomial (the other one, made monic, is the
gcd) or a nonzero constant (gcd 1).  A step of either rule is a unit multiple of the other's, so
both give the same sequence of degrees, the same number of steps and, made monic, the same gcd,
which is the oracle's; the number of steps stays within deg a + deg b + 2, the bound the host's
round count rests on."""
import numpy as np
import pytest

import oracle
from paper_1402_0264_gb300 import inputs


def trim(x):
    x = list(x)
    while x and x[-1] == 0:
        x.pop()
    return x


def run_steps(a, b, p, rule):
    """(the monic gcd as a list, degrees after each step, number of steps)."""
    a, b = trim(int(v) % p for v in a), trim(int(v) % p for v in b)
    unit = pow(2, -32, p) if rule == "mont" else 1
    degs, steps = [], 0
    while True:
        if not a or not b:
            g = a or b
            if not g:
                return [], degs, steps
            inv = pow(g[-1], p - 2, p)
            return [v * inv % p for v in g], degs, steps
        if len(a) == 1 or len(b) == 1:
            return [1], degs, steps
        red_a = len(a) >= len(b)
        r, d = (a, b) if red_a else (b, a)
        sh = len(r) - len(d)
        if rule == "paper":
            c1, c2 = 1, r[-1] * pow(d[-1], p - 2, p) % p
        else:
            c1, c2 = d[-1], r[-1]
        new = [c1 * v % p for v in r]
        for j, v in enumerate(d):
            new[j + sh] = (new[j + sh] - c2 * v) % p
        new = trim(v * unit % p for v in new)
        assert len(new) < len(r)          # the leading term is cancelled
        if red_a:
            a = new
        else:
            b = new
        steps += 1
        degs.append((len(a) - 1, len(b) - 1))


def cases():
    rng = np.random.default_rng(1406)
    out = []
    for p in (7681, 12289, inputs.P_DEFAULT):
        for da, db, dg in [(40, 30, 0), (40, 30, 7), (25, 25, 3), (1, 60, 0), (33, 33, 33), (50, 2, 1)]:
            g = list(rng.integers(0, p, dg + 1)); g[-1] = g[-1] or 1
            u = list(rng.integers(0, p, da - dg + 1)); u[-1] = u[-1] or 1
            v = list(rng.integers(0, p, db - dg + 1)); v[-1] = v[-1] or 1
            a = np.convolve(np.array(g, dtype=object), np.array(u, dtype=object)) % p
            b = np.convolve(np.array(g, dtype=object), np.array(v, dtype=object)) % p
            out.append((list(a), list(b), p))
        # sparse inputs whose degrees drop by more than one in a step, and exact multiples
        a = [0] * 30 + [1]; a[3] = 5
        b = [0] * 20 + [1]; b[0] = 2
        out.append((a, b, p))
        c = list(rng.integers(0, p, 12)); c[-1] = c[-1] or 1
        out.append((list(np.convolve(np.array(c, dtype=object), np.array([1, 2, 3], dtype=object)) % p), c, p))
    return out


@pytest.mark.parametrize("k", range(len(cases())))
def test_fraction_free_and_montgomery_steps_follow_the_paper(k):
    a, b, p = cases()[k]
    g0, degs0, n0 = run_steps(a, b, p, "paper")
    for rule in ("fraction_free", "mont"):
        g1, degs1, n1 = run_steps(a, b, p, rule)
        assert (degs1, n1) == (degs0, n0), rule
        assert g1 == g0, rule
    want = [int(v) for v in oracle.gcd(np.array(a, np.uint32), np.array(b, np.uint32), p)]
    assert g0 == want
    assert n0 <= (len(trim(a)) - 1) + (len(trim(b)) - 1) + 2


def test_special_cases_of_the_stop_rule():
    p = 7681
    assert run_steps([0, 0], [0], p, "mont")[0] == []
    assert run_steps([0, 0, 3], [0], p, "mont")[0] == [0, 0, 1]
    assert run_steps([5, 1, 4], [9], p, "mont")[0] == [1]             # a nonzero constant
    assert run_steps([2, 3, 1], [2, 3, 1], p, "mont") == ([2, 3, 1], [(-1, 2)], 1)   # a == b: one step
