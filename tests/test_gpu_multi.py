"""ncf_corr_batch_multi: several estimators of one device batch on one statistics
pass give exactly what separate ncf_corr_batch calls give (rectangle counts and
estimates identical, FP64 paths to the last bit of their summation order, the
FP32 form within its rounding)."""
import numpy as np
import pytest

from paper_2609_03866_b300 import api, synth
from tests._gpu import to_np

pytestmark = pytest.mark.gpu

OPTS = [dict(kernel="gaussian", h=0.5, path="spectral", precision="fp32"),
        dict(kernel="rectangle", h=0.5),
        dict(kernel="gaussian", h=0.5, path="spectral", precision="fp64", norm="lag0"),
        dict(kernel="gaussian", h=0.5, path="windowed", precision="fp64"),
        dict(kernel="rectangle", h=0.5, norm="lag0")]


def _check(multi, single, opt):
    if opt["kernel"] == "rectangle":
        assert np.array_equal(multi["count"], single["count"])
        assert np.array_equal(multi["c"], single["c"])
    else:
        tol = 1e-6 if opt.get("precision") == "fp32" else 1e-12
        assert np.max(np.abs(multi["c"] - single["c"])) < tol, opt


def test_multi_acf_batch_equals_separate_calls():
    w = synth.light_curves(B=40, n_lo=200, n_hi=20_000, K=48, seed=synth.BASE_SEED + 61)
    multi = [to_np(r) for r in api.corr_batch_multi(w.offs, w.t, w.x, w.lags, OPTS)]
    for m, o in zip(multi, OPTS):
        _check(m, to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, **o)), o)


def test_multi_ccf_equals_separate_calls():
    w = synth.ou_ccf(nA=8000, nB=6000, K=41)
    offs = np.array([0, w.t.size], dtype=np.int64)
    offs_y = np.array([0, w.s.size], dtype=np.int64)
    opts = OPTS
    multi = [to_np(r) for r in api.corr_batch_multi(offs, w.t, w.x, w.lags, opts, offs_y=offs_y, s=w.s, y=w.y)]
    for m, o in zip(multi, opts):
        _check(m, to_np(api.corr_batch(offs, w.t, w.x, w.lags, offs_y=offs_y, s=w.s, y=w.y, **o)), o)


def test_multi_rejects_bad_option_sets():
    w = synth.light_curves(B=3, n_lo=200, n_hi=2000, K=8, seed=synth.BASE_SEED + 62)
    with pytest.raises(api.NcfError) as e:
        api.corr_batch_multi(w.offs, w.t, w.x, w.lags, [OPTS[0], dict(kernel="gaussian", h=-1.0)])
    assert e.value.status == 1
    with pytest.raises(ValueError):
        api.corr_batch_multi(w.offs, w.t, w.x, w.lags, [])
