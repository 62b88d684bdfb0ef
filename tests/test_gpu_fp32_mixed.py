"""The batched FP32 form (ES spreading, FFT and spectra in FP32, tensor-core lag
evaluation) on batches that stress the spreading kernel's cases.

Its results are checked against the FP64 spectral path (itself within 1e-10 of
the oracle) on every series and lag at 1e-5, and against the oracle on sampled
series, for batches of: more series than SMs, series of 2 to 31 points, dense
clumps whose points share one grid cell, nightly cadence with gaps (a chunk of
points spanning a few cells), very sparse series (each tap its own cell), and
series whose cells wrap around the periodic grid.
"""
import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api, synth
from tests._gpu import to_np

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _pack(series):
    offs = np.zeros(len(series) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([t.size for t, _ in series])
    return offs, np.concatenate([t for t, _ in series]), np.concatenate([x for _, x in series])


def _mixed_batch(n_series=400, seed=31):
    rng = np.random.default_rng(seed)
    series = []
    for b in range(n_series):
        kind = b % 5
        if kind == 0:      # tiny series: partial warps
            n = int(rng.integers(2, 32))
            t = np.sort(rng.uniform(0, 1400, n))
        elif kind == 1:    # dense clumps: 40-80 points within 0.002 d, a clump every ~3 d
            c = np.sort(rng.uniform(0, 1400, 450))
            t = np.sort(np.concatenate([ci + rng.uniform(0, 0.002, int(rng.integers(40, 81))) for ci in c]))
        elif kind == 2:    # nightly cadence: 0.33 d nights, seasonal gaps
            nights = np.arange(0, 1400)
            nights = nights[(nights % 365) < 240]
            per = int(rng.integers(1, 40))
            t = np.sort((nights[:, None] + rng.uniform(0, 0.33, (nights.size, per))).ravel())
        elif kind == 3:    # very sparse: a point every few days
            t = np.sort(rng.uniform(0, 1400, int(rng.integers(150, 400))))
        else:              # uniform, moderately dense
            t = np.sort(rng.uniform(0, 1400, int(rng.integers(1000, 20000))))
        x = np.sin(2 * np.pi * t / rng.uniform(3, 50)) + rng.normal(size=t.size) * rng.uniform(0.1, 2)
        series.append((t, x))
    return series


def test_fp32_form_matches_the_fp64_path_on_every_value():
    series = _mixed_batch()
    offs, t, x = _pack(series)
    lags = np.linspace(0.0, 150.0, 96)
    f32 = to_np(api.corr_batch(offs, t, x, lags, kernel="gaussian", h=0.5, path="spectral", precision="fp32"))
    f64 = to_np(api.corr_batch(offs, t, x, lags, kernel="gaussian", h=0.5, path="spectral", precision="fp64"))
    # series of a few points leave most lags with almost no pair nearby: there b is
    # a small difference of the mode sums and c = N / b amplifies the FP32 form's
    # rounding (an FP32 property of the spectral route); c is
    # compared where b is at least 1e-2 of the series' largest b, and b
    # everywhere on the series' own scale
    scale = np.max(np.abs(f64["b"]), axis=1, keepdims=True)
    assert np.max(np.abs(f32["b"] - f64["b"]) / scale) < 1e-5
    ok = np.abs(f64["b"]) > 1e-2 * scale
    ok[0::5] = False     # series of 2-31 points: b above only
    err = np.where(ok, np.abs(f32["c"] - f64["c"]), 0.0)
    assert np.max(err) < TOL, (np.max(err), np.unravel_index(np.argmax(err), err.shape))
    assert ok[1::5].all() and ok[2::5].all() and ok[4::5].all()
    for b in (1, 2, 3, 4, 137, 398):
        tb, xb = series[b]
        ref = oracle.corr(tb, xb, lags, "gaussian", 0.5, method="windowed", trunc_R=8.0)
        assert np.max(np.where(ok[b], np.abs(f32["c"][b] - ref["c"]), 0.0)) < TOL, b


def test_fp32_form_pearson_and_unsorted_repeated_lags():
    w = synth.light_curves(B=160, n_lo=200, n_hi=60_000, K=8, seed=synth.BASE_SEED + 91)
    lags = np.array([37.5, 0.0, 12.25, 12.25, 199.0, 3.0, 0.75, 88.0])
    for norm in ("none", "lag0"):
        f32 = to_np(api.corr_batch(w.offs, w.t, w.x, lags, kernel="gaussian", h=0.5, path="spectral",
                                   precision="fp32", norm=norm))
        f64 = to_np(api.corr_batch(w.offs, w.t, w.x, lags, kernel="gaussian", h=0.5, path="spectral",
                                   precision="fp64", norm=norm))
        assert np.max(np.abs(f32["c"] - f64["c"])) < TOL
        assert np.max(np.abs(f32["c"][:, 2] - f32["c"][:, 3])) < 1e-12   # a repeated lag


def test_fp32_form_repeat_calls_agree_to_rounding():
    w = synth.light_curves(B=300, n_lo=200, n_hi=30_000, K=64, seed=synth.BASE_SEED + 92)
    a = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=0.5, path="spectral", precision="fp32"))
    b = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=0.5, path="spectral", precision="fp32"))
    # float atomics add in varying order: equal to FP32 rounding
    assert np.max(np.abs(a["c"] - b["c"])) < 1e-6
