"""Empty windows in the exact rectangle scan (Algorithms 6 and 8).

The points-on-lanes scan decides, per lag and per slot of 32 consecutive outer
points, whether every window of the slot is empty, and then leaves the slot's
batch out: the count and the window sum of an empty window are 0 exactly.  The
cases below put many windows into seasonal gaps, past the end of the data and
between the disjoint seasons of a CCF pair.  Every scan variant (the lags-on-lanes
variants evaluate every window) must give the same counts and numerators, equal
to the FP64 oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api, synth
from tests._gpu import max_abs, to_np
from tests.test_gpu_rect_variants import all_variants

pytestmark = pytest.mark.gpu


def test_lags_into_seasonal_gaps_and_past_the_end():
    """Light curves (four 243-day seasons) at lags up to 1400 d: most windows of
    the long lags fall into the 122-day gaps or after the last season."""
    w = synth.light_curves(B=6, n_lo=20_000, n_hi=120_000, K=96, max_lag=1400.0, seed=synth.BASE_SEED + 31)
    got = all_variants(lambda: api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="rectangle", h=0.5))
    rng = np.random.default_rng(31)
    for b in range(w.B):
        sl = slice(int(w.offs[b]), int(w.offs[b + 1]))
        ks = np.sort(rng.choice(w.lags.size, 12, replace=False))
        ref = oracle.corr(w.t[sl], w.x[sl], w.lags[ks], "rectangle", 0.5, method="windowed")
        assert np.array_equal(got["count"][b, ks], ref["count"]), b
        assert max_abs(got["c"][b, ks], ref["c"]) < 1e-10, b
    # past the last season (separations of more than 1338.5 d) no lag has a pair
    assert np.all(got["count"][:, w.lags > 1339.0] == 0)


def test_every_window_empty():
    """Lags beyond the span of the data: no pair at any lag, count 0 and c 0."""
    w = synth.light_curves(B=3, n_lo=5_000, n_hi=60_000, K=40, seed=synth.BASE_SEED + 32)
    lags = np.linspace(1600.0, 1700.0, 40)  # four seasons end before day 3 * 365 + 243
    got = all_variants(lambda: api.corr_batch(w.offs, w.t, w.x, lags, kernel="rectangle", h=0.5))
    assert np.all(got["count"] == 0)
    for b in range(w.B):
        sl = slice(int(w.offs[b]), int(w.offs[b + 1]))
        ref = oracle.corr(w.t[sl], w.x[sl], lags, "rectangle", 0.5, method="windowed")
        assert np.array_equal(got["count"][b], ref["count"])
        assert max_abs(got["c"][b], ref["c"]) == 0.0


def test_ccf_with_disjoint_seasons():
    """x observed in years 0 and 2, y in years 1 and 3 (dense nights): at lags
    near 0 every window is empty; near +-365 d the seasons meet."""
    rng = np.random.default_rng(33)

    def seasons(years, per_night):
        nights = np.concatenate([365.0 * yr + np.arange(0, 200) for yr in years])
        return np.sort((nights[:, None] + rng.uniform(0.0, 0.33, (nights.size, per_night))).ravel())

    t = seasons((0, 2), 60)
    s = seasons((1, 3), 45)
    x = np.sin(t / 9.0) + rng.normal(size=t.size)
    y = np.sin(s / 9.0) + rng.normal(size=s.size)
    lags = np.linspace(-500.0, 500.0, 41)
    got = all_variants(lambda: api.corr(t, x, lags, kernel="rectangle", h=0.5, s=s, y=y))
    ref = oracle.corr(t, x, lags, "rectangle", 0.5, s=s, y=y, method="windowed")
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10
    assert np.sum(ref["count"] == 0) >= 5 and np.sum(ref["count"] > 0) >= 5


def test_pearson_normalisation_with_empty_lags():
    """The lag-0 (Pearson) scale is taken from the lag-0 window, which is never
    empty for an ACF; lags whose windows are all empty keep c = 0."""
    w = synth.light_curves(B=4, n_lo=3_000, n_hi=40_000, K=30, seed=synth.BASE_SEED + 34)
    lags = np.concatenate([np.linspace(0.0, 20.0, 15), np.linspace(1600.0, 1650.0, 15)])
    got = to_np(api.corr_batch(w.offs, w.t, w.x, lags, kernel="rectangle", h=0.5, norm="lag0"))
    for b in range(w.B):
        sl = slice(int(w.offs[b]), int(w.offs[b + 1]))
        ref = oracle.corr(w.t[sl], w.x[sl], lags, "rectangle", 0.5, method="windowed", norm="lag0")
        assert np.array_equal(got["count"][b], ref["count"])
        assert max_abs(got["c"][b], ref["c"]) < 1e-10
        assert np.all(got["c"][b, 15:] == 0.0)
