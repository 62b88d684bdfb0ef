"""The empty-window rule of the points-on-lanes rectangle scan, emulated on the CPU.

The scan works on fixed-point keys T (times scaled to integers) coarsened by a
shift: c = ((T - base) >> sh) - vmin for a key, s_j = (S_j - S0) >> sh for an
outer point, and per lag the offsets
    Lx = ((S0 + dl - eta - base) >> sh) - vmin,  Lw = ((S0 + du + eta - base) >> sh) + 2 - vmin,
where [S_j + dl, S_j + du] is the window of point j in fixed point and eta the
margin inside which the FP64 predicate decides (Algorithms 6 and 8).  For a slot
of outer points with coarse offsets in [lo, hi] the kernel leaves the slot out
when the first key with c >= lo + Lx has c >= hi + Lw.  The rule must be
conservative: whenever it fires, no key lies in [S_j + dl - eta, S_j + du + eta]
for any point j of the slot, so every window is empty whatever the FP64
predicate decides.  This file checks that by brute force on random and
clustered inputs, with the kernel's integer formulas written out here (Python
integers: >> is the same floor shift as the kernel's on int64).
"""
import bisect

import numpy as np


def rule_fires(T, S, dl, du, eta, sh):
    S0 = S[0]
    base = S0 + dl - eta            # the sub-group's lowest lower bound (one lag here)
    vmin = 0 + ((S0 + dl - eta - base) >> sh)
    c = [((t - base) >> sh) - vmin for t in T]
    s = [(x - S0) >> sh for x in S]
    Lx = ((S0 + dl - eta - base) >> sh) - vmin
    Lw = ((S0 + du + eta - base) >> sh) + 2 - vmin
    lo, hi = min(s), max(s)
    e = bisect.bisect_left(c, lo + Lx)
    return e == len(c) or c[e] >= hi + Lw


def truly_empty(T, S, dl, du, eta):
    for x in S:
        a = bisect.bisect_left(T, x + dl - eta)
        if a < len(T) and T[a] <= x + du + eta:
            return False
    return True


def check(rng, clustered):
    sh = int(rng.integers(0, 12))
    eta = int(rng.integers(0, 1 << 8))
    if clustered:  # nights: keys in short clusters with long gaps, as in the light curves
        nights = np.sort(rng.choice(400, 60, replace=False))
        T = np.sort((nights[:, None] * 4096 + rng.integers(0, 1300, (60, 20))).ravel())
    else:
        T = np.sort(rng.integers(0, 1 << 20, int(rng.integers(1, 400))))
    T = [int(v) for v in T]
    j0 = int(rng.integers(0, len(T)))
    S = sorted(int(v) for v in (T[j0] + rng.integers(0, 1 << int(rng.integers(1, 14)), 32)))
    dl = int(rng.integers(-(1 << 16), 1 << 16))
    du = dl + int(rng.integers(0, 1 << 12))
    fired = rule_fires(T, S, dl, du, eta, sh)
    if fired:
        assert truly_empty(T, S, dl, du, eta), (sh, eta, dl, du)
    return fired, truly_empty(T, S, dl, du, eta)


def test_rule_is_conservative_on_random_and_clustered_keys():
    rng = np.random.default_rng(20260903)
    fired = empty = 0
    for i in range(3000):
        f, e = check(rng, clustered=bool(i % 2))
        fired += f
        empty += e
    # the rule is exercised, and it catches most of the empty slots
    assert fired > 300 and fired >= 0.5 * empty


def test_rule_on_hand_made_edges():
    # a key exactly at a window edge of the first and of the last point: never skipped
    S = [1000, 1010, 1020]
    for T in ([1000 + 50], [1020 + 80], [1000 + 49], [1020 + 81]):
        for sh in (0, 3, 6):
            if not truly_empty(T, S, 50, 60, 0):
                assert not rule_fires(T, S, 50, 60, 0, sh), (T, sh)
    # keys far outside every window: skipped at shift 0
    assert rule_fires([0, 1, 5000], S, 50, 60, 0, 0)
