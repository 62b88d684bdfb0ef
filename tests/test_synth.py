"""The seeded input generators shared by the oracle checks, the GPU parity tests
and the benchmark: deterministic for a seed, with the structure each workload
promises (sorted times per series, CSR offsets, sizes, seasonal gaps, MJD-scale
times, and the OU pair's delay)."""
import numpy as np

import oracle
from paper_2609_03866_b300 import synth


def test_light_curves_are_deterministic_and_well_formed():
    a = synth.light_curves(B=24, n_lo=200, n_hi=20_000, K=16, seed=synth.BASE_SEED + 3, threads=2)
    b = synth.light_curves(B=24, n_lo=200, n_hi=20_000, K=16, seed=synth.BASE_SEED + 3, threads=5)
    assert np.array_equal(a.offs, b.offs) and np.array_equal(a.t, b.t) and np.array_equal(a.x, b.x)
    c = synth.light_curves(B=24, n_lo=200, n_hi=20_000, K=16, seed=synth.BASE_SEED + 4)
    assert not np.array_equal(a.t[:100], c.t[:100])
    sizes = np.diff(a.offs)
    assert a.offs[0] == 0 and np.all(sizes >= 200) and np.all(sizes <= 20_000)
    assert np.array_equal(a.lags, np.linspace(0.0, 200.0, 16))
    assert np.all(np.isfinite(a.t)) and np.all(np.isfinite(a.x))
    for k in range(a.B):
        t, x, _, _ = a.series(k)
        assert np.all(np.diff(t) >= 0.0)
        assert t[-1] - t[0] < 4 * 365.0 and np.max(np.diff(t)) > 60.0   # four seasons with gaps
        assert np.std(x) > 0.0


def test_ou_pair_is_sorted_and_y_lags_x_by_the_delay():
    w = synth.ou_ccf(nA=20_000, nB=16_000, K=41, delay=15.0)
    assert np.all(np.diff(w.t) >= 0) and np.all(np.diff(w.s) >= 0)
    assert (w.t.size, w.s.size) == (20_000, 16_000)
    assert np.array_equal(w.lags, np.linspace(-100.0, 100.0, 41))
    # each year's last 120 days unobserved
    assert np.max(np.diff(w.t)) > 100.0 and np.max(np.diff(w.s)) > 100.0
    lags = np.arange(0.0, 31.0)
    r = oracle.corr(w.t, w.x, lags, "rectangle", 0.5, s=w.s, y=w.y, method="windowed")
    assert abs(lags[int(np.argmax(r["c"]))] - 15.0) <= 1.0


def test_ar1_and_quasi_periodic_workloads():
    w = synth.ar1_acf(n=500, K=11)
    assert w.t.size == 500 and np.all(np.diff(w.t) >= 0) and w.t.min() >= 0 and w.t.max() <= 1000
    assert np.array_equal(w.lags, np.linspace(0.0, 100.0, 11))
    q = synth.quasi_periodic(n=20_000, K=7)
    assert np.all(np.diff(q.t) >= 0) and q.t.min() >= 60000.0 and q.t.max() <= 80000.0
    assert np.array_equal(synth.quasi_periodic(n=20_000, K=7).x, q.x)
