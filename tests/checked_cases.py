"""Small cases of every path run through the range-checked build (-DPOLYMUL_CHECKED), in a process
of its own: `python -m tests.checked_cases` with POLYMUL_LIBRARY naming that build.  Every result
must equal the oracle's and leave the status word clear (no guarded index was out of range); then a
word >= p in an input must set PM_ERR_RANGE.  Prints one line and exits 0 when all hold."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1402_0264_gb300 import inputs  # noqa: E402
from paper_1402_0264_gb300 import polymul as pm  # noqa: E402
from tests.gpuhelp import assert_equal, dev, dev64, host  # noqa: E402

P = inputs.P_DEFAULT


def clean(what):
    st = pm.sync_status()
    assert st == 0, f"{what}: status {pm.STATUS.get(st, st)}"


def main():
    assert "checked" in pm.LIB_PATH, pm.LIB_PATH
    # plain, several s, both operand orders, one tile and many
    for da, db, s in ((0, 0, 1), (700, 500, 8), (300, 2500, 4), (4096, 4096, 16), (9000, 33, 64), (2047, 2047, 32)):
        a, b = inputs.poly_pair(da, db, inputs.SEED_BASE + 900 + da + db)
        assert_equal(host(pm.plain(dev(a), dev(b), s=s)), oracle.polymul(a, b, P), f"plain {da}x{db} s={s}")
        clean("plain")
    a, b = inputs.poly_pair(3000, 1000, inputs.SEED_BASE + 901)
    assert_equal(host(pm.plain_ell(dev(a), dev(b), 8, 128)), oracle.polymul(a, b, P), "plain_ell")
    clean("plain_ell")
    # batched: warp-level form, CTA form, tensor cores (one and several K-groups)
    packed = inputs.packed_batch(np.array([3, 100, 700, 2048]), np.array([50, 9, 500, 2048]), inputs.SEED_BASE + 902)
    want = oracle.polymul_batch(*packed[:4], packed[4], P)
    t = [dev(packed[0]), dev64(packed[1]), dev(packed[2]), dev64(packed[3]), dev64(packed[4])]
    for mode, s, md in ((pm.PM_PLAIN, 8, 2048), (pm.PM_PLAIN, 64, 5000), (pm.PM_TENSOR, 0, 2048)):
        assert_equal(host(pm.batched(*t, max_deg=md, mode=mode, s=s, total=int(packed[4][-1]))), want,
                     f"batched mode {mode} s {s}")
        clean("batched")
    big = inputs.packed_batch(np.array([8191, 100]), np.array([5000, 8191]), inputs.SEED_BASE + 903)
    tb = [dev(big[0]), dev64(big[1]), dev(big[2]), dev64(big[3]), dev64(big[4])]
    assert_equal(host(pm.batched(*tb, max_deg=8191, mode=pm.PM_TENSOR, total=int(big[4][-1]))),
                 oracle.polymul_batch(*big[:4], big[4], P), "tensor K-groups")
    clean("tensor")
    # transforms: one CTA, and the four-step passes with 16 and 8 columns
    for na, nb in ((300, 200), (6000, 5000), (1 << 20, 1 << 20)):
        a, b = inputs.poly_pair(na - 1, nb - 1, inputs.SEED_BASE + 904 + na)
        got = host(pm.ntt(dev(a), dev(b)))
        if na < 10000:
            assert_equal(got, oracle.polymul(a, b, P), f"ntt {na}")
        else:
            k = np.array([0, 1, 777, na, na + nb - 2])
            assert_equal(got[k], [oracle.coeff(a, b, P, int(x)) for x in k], f"ntt {na} sampled")
        clean("ntt")
    # division and gcd
    a, b = inputs.poly_pair(3000, 1000, inputs.SEED_BASE + 905)
    b[-1] = max(int(b[-1]), 1)
    q, r = pm.divide(dev(a), dev(b), s=128)
    qw, rw = oracle.divide(a, b, P)
    assert_equal(host(q), qw, "division q")
    assert_equal(host(r), rw, "division r")
    clean("division")
    g, u, v = inputs.gcd_cofactors(60, 700, 500, inputs.SEED_BASE + 906)
    ga, gb = oracle.polymul(g, u, P), oracle.polymul(g, v, P)
    for s in (1, 64, 256):
        assert_equal(host(pm.gcd(dev(ga), dev(gb), s=s)), oracle.gcd(ga, gb, P), f"gcd s={s}")
        clean("gcd")
    # a word >= p: the checked build's input scan reports PM_ERR_RANGE
    a, b = inputs.poly_pair(500, 400, inputs.SEED_BASE + 907)
    a[123] = P
    pm.plain(dev(a), dev(b), s=8)
    assert pm.sync_status() == 2, "plain: a word >= p was not reported"
    pm.ntt(dev(b), dev(a))
    assert pm.sync_status() == 2, "ntt: a word >= p was not reported"
    bad = inputs.packed_batch(np.array([10, 20]), np.array([30, 40]), inputs.SEED_BASE + 908)
    bad[2][35] = 0xFFFFFFFF
    pm.batched(dev(bad[0]), dev64(bad[1]), dev(bad[2]), dev64(bad[3]), dev64(bad[4]), max_deg=40, mode=pm.PM_PLAIN,
               total=int(bad[4][-1]))
    assert pm.sync_status() == 2, "batched: a word >= p was not reported"
    b2 = b.copy()
    b2[-1] = P + 5
    pm.divide(dev(a[:450] % P), dev(b2))
    assert pm.sync_status() == 2, "division: a word >= p was not reported"
    # and the next clean call is clean
    a, b = inputs.poly_pair(500, 400, inputs.SEED_BASE + 909)
    assert_equal(host(pm.plain(dev(a), dev(b), s=8)), oracle.polymul(a, b, P), "after the range reports")
    clean("after")
    print("checked build ok", flush=True)


if __name__ == "__main__":
    main()
