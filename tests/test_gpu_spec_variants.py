"""The autotuner's FP32 spectral shapes: the spreading (CTAs of 4096 or 2048
points; tile sums in FP32 or in fixed point), the FFT of an ACF grid of up to
2^14 cells in shared memory (fused with its spectrum) or as global passes, and
the mode-to-lag contraction on tensor cores or on the FP32 pipe.

Each of the sixteen shapes, pinned with NCF_SPEC_VARIANT, and the shape the tuner
picks by itself must match the FP64 spectral path (within 1e-10 of the oracle)
at the FP32 form's 1e-5 on every series and lag, for a light-curve batch and a
batch of cross-correlations (where the contraction and the spreading vary).
"""
import os

import numpy as np
import pytest

from paper_2609_03866_b300 import api, synth
from tests._gpu import to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _pinned(v, fn):
    old = os.environ.get("NCF_SPEC_VARIANT")
    if v is None:
        os.environ.pop("NCF_SPEC_VARIANT", None)
    else:
        os.environ["NCF_SPEC_VARIANT"] = str(v)
    try:
        return fn()
    finally:
        if old is None:
            os.environ.pop("NCF_SPEC_VARIANT", None)
        else:
            os.environ["NCF_SPEC_VARIANT"] = old


@pytest.mark.parametrize("variant", list(range(16)) + [None])
def test_acf_batch_every_shape_matches_fp64(variant):
    w = synth.light_curves(B=160, n_lo=200, n_hi=40_000, K=130, seed=77)
    ref = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=0.5, path="spectral",
                               precision="fp64"))
    got = _pinned(variant, lambda: to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=0.5,
                                                        path="spectral", precision="fp32")))
    assert np.all(np.isfinite(got["c"]))
    assert np.max(np.abs(got["c"] - ref["c"])) < TOL
    assert np.max(np.abs(got["b"] / ref["b"] - 1.0)) < 1e-4


@pytest.mark.parametrize("variant", [0, 2, 8, 14])
def test_ccf_batch_contractions_and_spreadings_match_fp64(variant):
    rng = np.random.default_rng(5)
    B = 24
    xs, ys = [], []
    for b in range(B):
        w = synth.ou_ccf(nA=int(rng.integers(500, 4000)), nB=int(rng.integers(500, 4000)), K=41, seed=100 + b)
        xs.append((w.t, w.x))
        ys.append((w.s, w.y))
        lags = w.lags
    ox = np.concatenate([[0], np.cumsum([t.size for t, _ in xs])]).astype(np.int64)
    oy = np.concatenate([[0], np.cumsum([s.size for s, _ in ys])]).astype(np.int64)
    t = np.concatenate([a for a, _ in xs]); x = np.concatenate([b for _, b in xs])
    s = np.concatenate([a for a, _ in ys]); y = np.concatenate([b for _, b in ys])
    kw = dict(kernel="gaussian", h=0.5, offs_y=oy, s=s, y=y, path="spectral")
    ref = to_np(api.corr_batch(ox, t, x, lags, precision="fp64", **kw))
    got = _pinned(variant, lambda: to_np(api.corr_batch(ox, t, x, lags, precision="fp32", **kw)))
    assert np.max(np.abs(got["c"] - ref["c"])) < TOL


def test_last_tuning_reports_the_shapes_used():
    w = synth.light_curves(B=40, n_lo=500, n_hi=5000, K=20, seed=78)
    ctx = api.Context()
    try:
        for v in range(16):
            _pinned(v, lambda: api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=0.5,
                                              path="spectral", precision="fp32", ctx=ctx))
            tu = ctx.last_tuning()
            assert tu["fft_variant"] == (v & 1) and tu["contract_variant"] == ((v >> 1) & 1), (v, tu)
            assert tu["spread_variant"] == (v >> 2), (v, tu)
        _pinned(1, lambda: api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="rectangle", h=0.5, ctx=ctx))
        assert ctx.last_tuning()["rect_variant"] in (0, 1, 2, 3)
    finally:
        ctx.close()


@pytest.mark.parametrize("variant", [4, 12])
def test_fixed_point_tiles_with_outliers(variant):
    """Fixed-point tile sums take their scale from the chunk's sum of |x_std|, so a
    few extreme values coarsen it for every other point of the chunk: light curves
    with five points per series raised 1000-fold (a 1000-sigma outlier next to
    ordinary values), FP32 sums (variant 4) and fixed-point sums (12), both
    against the FP64 spectral path at the FP32 form's 1e-5."""
    w = synth.light_curves(B=48, n_lo=2000, n_hi=60_000, K=90, seed=91)
    x = w.x.copy()
    rng = np.random.default_rng(92)
    for b in range(w.B):
        a, e = int(w.offs[b]), int(w.offs[b + 1])
        x[rng.choice(np.arange(a, e), 5, replace=False)] *= 1000.0
    ref = to_np(api.corr_batch(w.offs, w.t, x, w.lags, kernel="gaussian", h=0.5, path="spectral",
                               precision="fp64"))
    got = _pinned(variant, lambda: to_np(api.corr_batch(w.offs, w.t, x, w.lags, kernel="gaussian", h=0.5,
                                                        path="spectral", precision="fp32")))
    assert np.all(np.isfinite(got["c"]))
    assert np.max(np.abs(got["c"] - ref["c"])) < TOL
