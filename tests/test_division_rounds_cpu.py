"""The round structure of the GPU division, checked on the CPU against the oracle (no kernel runs).

Section 3's optimized division runs s division steps per kernel call.  In each round the head
(the s leading coefficients of the current remainder) is carried through the s steps one at a
time, which gives the round's s quotient coefficients; every position below the head then
receives all s steps at once, r[x] -= sum_k q_k b[x - (t - k) + deg b] with t the round's top
index, because the steps' updates are linear and commute.  The emulation below does exactly that
and must give the oracle's quotient and remainder for every s, including rounds shorter than s
at the end."""
import numpy as np
import pytest

import oracle


def divide_in_rounds(a, b, p, s):
    a = [int(v) % p for v in a]
    b = [int(v) % p for v in b]
    n, m = len(a), len(b)
    db = m - 1
    inv = pow(b[-1], p - 2, p)
    r = list(a)
    q = [0] * (n - m + 1)
    top = n - 1
    while top >= db:
        steps = min(s, top - db + 1)
        lo = top - steps + 1                    # the head: positions lo .. top
        head = r[lo: top + 1]
        qs = []
        for k in range(steps):                   # one step at a time on the head
            t = top - k
            qk = head[t - lo] * inv % p
            qs.append(qk)
            for j in range(1, m):                # head entries below t
                x = t - j
                if x >= lo:
                    head[x - lo] = (head[x - lo] - qk * b[db - j]) % p
            head[t - lo] = 0
        for k, qk in enumerate(qs):
            q[top - k - db] = qk
        for x in range(max(0, lo - db), lo):     # the body: all of the round's steps at once
            acc = 0
            for k, qk in enumerate(qs):
                j = x - (top - k) + db
                if 0 <= j <= db:
                    acc += qk * b[j]
            r[x] = (r[x] - acc) % p
        for x in range(lo, top + 1):
            r[x] = 0
        top = lo - 1
    return q, r[:db]


@pytest.mark.parametrize("p", [7681, 469762049, (1 << 30) - 35])
@pytest.mark.parametrize("n,m", [(1, 1), (5, 5), (40, 3), (100, 37), (130, 129), (64, 1)])
@pytest.mark.parametrize("s", [1, 3, 8, 32, 256])
def test_rounds_match_the_oracle(p, n, m, s):
    rng = np.random.default_rng(n * 1000 + m * 10 + s)
    a = rng.integers(0, p, n).astype(np.uint64)
    b = rng.integers(0, p, m).astype(np.uint64)
    b[-1] = b[-1] or 1
    q, r = divide_in_rounds(a, b, p, s)
    wq, wr = oracle.divide(a.astype(np.uint32), b.astype(np.uint32), p)
    assert q == [int(v) for v in wq]
    assert r == [int(v) for v in wr]
