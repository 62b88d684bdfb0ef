"""Every rectangle-scan variant the autotuner can pick gives the same exact
pair counts and numerators, equal to the FP64 oracle (Algorithms 6 and 8).

Variants 0-2 put lags on lanes (runs of 16 / 32 / 64 outer points); variant 3
puts outer points on lanes with a rank table, splits a lag group into
sub-groups when its key union does not fit shared memory, splits the outer
points of a tile (at its widest time gap, else in the middle) when one lag's
union does not fit, and runs a lag on the global keys when a single outer
point's window fills half the staging area.  The cases below reach each of
those branches.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api, synth
from tests._gpu import max_abs, to_np

pytestmark = pytest.mark.gpu
VARIANTS = (0, 1, 2, 3)


def run_variant(v, fn):
    old = os.environ.get("NCF_RECT_VARIANT")
    os.environ["NCF_RECT_VARIANT"] = str(v)
    try:
        return fn()
    finally:
        if old is None:
            del os.environ["NCF_RECT_VARIANT"]
        else:
            os.environ["NCF_RECT_VARIANT"] = old


def all_variants(fn):
    outs = [to_np(run_variant(v, fn)) for v in VARIANTS]
    for o in outs[1:]:
        assert np.array_equal(o["count"], outs[0]["count"])
        assert np.array_equal(o["c"], outs[0]["c"])      # bit-identical: exact integer sums
    return outs[0]


def test_dense_light_curves_lag_subgroups():
    """Dense series (the key union of 32 lags exceeds the staging area)."""
    w = synth.light_curves(B=3, n_lo=120_000, n_hi=200_000, K=96, seed=synth.BASE_SEED + 17)
    got = all_variants(lambda: api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="rectangle", h=0.5))
    rng = np.random.default_rng(1)
    for b in range(w.B):
        sl = slice(int(w.offs[b]), int(w.offs[b + 1]))
        ks = rng.choice(w.lags.size, 6, replace=False)
        ref = oracle.corr(w.t[sl], w.x[sl], w.lags[ks], "rectangle", 0.5, method="windowed")
        assert np.array_equal(got["count"][b, ks], ref["count"])
        assert max_abs(got["c"][b, ks], ref["c"]) < 1e-10


def test_sparse_outer_dense_inner_ccf_middle_splits():
    """CCF whose outer series is sparse over a long span and inner series dense:
    a single lag's union exceeds the staging area and the tile, with no
    dominant gap, is split in the middle down to small segments."""
    rng = np.random.default_rng(2)
    t = np.sort(rng.uniform(0, 3000, 150_000))
    x = rng.normal(size=t.size)
    s = np.sort(rng.uniform(0, 3000, 2500))
    y = rng.normal(size=s.size)
    lags = np.linspace(-40, 40, 37)
    got = all_variants(lambda: api.corr(t, x, lags, kernel="rectangle", h=0.75, s=s, y=y))
    ref = oracle.corr(t, x, lags, "rectangle", 0.75, s=s, y=y, method="windowed")
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10


def test_dense_seasons_across_a_gap_split_at_the_gap():
    """Two dense observing seasons 120 days apart: the tile holding the season
    boundary spans the gap, and at lags that carry its windows into the other
    season one lag's union far exceeds the staging area; the split falls at the
    gap.  Counts are exact and equal the oracle's at every lag."""
    rng = np.random.default_rng(21)
    nights = np.concatenate([np.arange(0, 60), np.arange(180, 240)]).astype(np.float64)
    t = np.sort((nights[:, None] + rng.uniform(0.0, 0.3, (nights.size, 200))).ravel())
    x = np.sin(t / 7.0) + rng.normal(size=t.size)
    lags = np.linspace(0.0, 200.0, 64)
    got = all_variants(lambda: api.corr(t, x, lags, kernel="rectangle", h=0.5))
    ref = oracle.corr(t, x, lags, "rectangle", 0.5, method="windowed")
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10


def test_wide_windows_global_path():
    """A window of 2h = 40 days over 100 points a day holds 4000 keys, more than
    half the staging area: such lags run on the global keys."""
    rng = np.random.default_rng(22)
    t = np.sort(rng.uniform(0.0, 400.0, 40_000))
    x = rng.normal(size=t.size)
    s = np.sort(rng.uniform(0.0, 400.0, 3000))
    y = rng.normal(size=s.size)
    lags = np.linspace(-50.0, 50.0, 21)
    got = all_variants(lambda: api.corr(t, x, lags, kernel="rectangle", h=20.0, s=s, y=y))
    ref = oracle.corr(t, x, lags, "rectangle", 20.0, s=s, y=y, method="windowed")
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10


def test_boundary_ties_unsorted_lags_tiny_width():
    """Integer grid: window bounds land on sample times (FP64 band); unsorted
    and repeated lags; a half-width far below the spacing (empty windows,
    hi < lo after the band)."""
    rng = np.random.default_rng(3)
    t = np.sort(rng.choice(60_000, 9000, replace=False)).astype(np.float64)
    x = rng.normal(size=t.size)
    lags = np.array([7.0, -3.0, 0.0, 12.0, 7.0, 1.0, -15.0, 40.0] * 5)
    for h in (1.0, 0.5, 1e-9):
        got = all_variants(lambda: api.corr(t, x, lags, kernel="rectangle", h=h))
        ref = oracle.corr(t, x, lags, "rectangle", h, method="windowed")
        assert np.array_equal(got["count"], ref["count"])
        assert max_abs(got["c"], ref["c"]) < 1e-10
    s = t[::3] + 2.0
    got = all_variants(lambda: api.corr(t, x, lags, kernel="rectangle", h=1.0, s=s, y=x[::3]))
    ref = oracle.corr(t, x, lags, "rectangle", 1.0, s=s, y=x[::3], method="windowed")
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10


def test_ragged_batch_small_and_large_series():
    """Series from 2 to 30 000 points in one batch (partial tiles, lanes with
    no outer point, lag groups cut at K)."""
    sizes = [2, 3, 31, 33, 2047, 2049, 30_000, 500]
    w = synth.light_curves(B=len(sizes), K=45, sizes=sizes, seed=synth.BASE_SEED + 5)
    got = all_variants(lambda: api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="rectangle", h=0.5))
    for b in range(w.B):
        sl = slice(int(w.offs[b]), int(w.offs[b + 1]))
        ref = oracle.corr(w.t[sl], w.x[sl], w.lags, "rectangle", 0.5, method="windowed")
        assert np.array_equal(got["count"][b], ref["count"])
        assert max_abs(got["c"][b], ref["c"]) < 1e-10


@pytest.mark.parametrize("B,K", [(64, 256), (1, 1), (3, 257), (128, 33)])
def test_workspace_sizes_for_any_batch_and_lag_count(B, K):
    """Device workspace estimates hold for every (B, K): lag copies, per-series
    scale arrays and tile tables all fit (no NCF_ENOMEM)."""
    w = synth.light_curves(B=B, n_lo=200, n_hi=3000, K=K, seed=synth.BASE_SEED + B + K)
    for norm in ("none", "lag0"):
        r = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="rectangle", h=0.5, norm=norm))
        assert r["c"].shape == (B, K) and np.all(np.isfinite(r["c"]))
    r = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=0.5, path="windowed"))
    assert np.all(np.isfinite(r["c"]))
    for prec in ("fp64", "fp32"):
        r = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=0.5, path="spectral",
                                 precision=prec))
        assert np.all(np.isfinite(r["c"]))


def test_same_call_twice_gives_identical_results():
    # the scan's sums are exact integers added with integer atomics: no run-to-run
    # difference is allowed, in any variant
    w = synth.light_curves(B=96, K=40, seed=synth.BASE_SEED + 9)
    for v in VARIANTS:
        a = to_np(run_variant(v, lambda: api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="rectangle", h=0.5)))
        b = to_np(run_variant(v, lambda: api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="rectangle", h=0.5)))
        for key in ("count", "b", "c"):
            assert np.array_equal(a[key], b[key]), (v, key)
