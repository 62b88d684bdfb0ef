"""One long series split by outer index (shard.split_series) on the GPU library,
the ranges evaluated one after another on this GPU through ncf_corr_pooled and
their statistics pooled from ncf_series_stats: the same result as the unsplit
call, pair counts bit-exact, c within 1e-10 (FP64) or 1e-5 (FP32 form).  The
multi-rank reduction itself is tested on gloo ranks (test_shard_gloo.py)."""
import numpy as np
import pytest

from paper_2609_03866_b300 import api, shard, synth

pytestmark = pytest.mark.gpu


def _run(t, x, lags, world, s=None, y=None, **kw):
    ev = shard.gpu_evaluator(api, **kw)
    return shard.split_series(t, x, lags, ev, shard.gpu_summarizer(api), rank=None, world=world, s=s, y=y,
                              kernel=kw.get("kernel", "rectangle"), h=kw["h"], path=kw.get("path", "auto"),
                              trunc_R=kw.get("trunc_R", 0.0))


@pytest.mark.parametrize("world", [1, 2, 3, 7])
def test_split_ccf_seasonal_ou(world):
    w = synth.ou_ccf()                           # 1e5 x 8e4 points, 200 lags
    for kw, tol in ((dict(kernel="rectangle", h=0.5), 1e-10),
                    (dict(kernel="gaussian", h=0.5, path="windowed"), 1e-10),
                    (dict(kernel="gaussian", h=0.5, path="spectral"), 1e-10)):
        ref = {k: v.cpu().numpy() for k, v in api.corr(w.t, w.x, w.lags, s=w.s, y=w.y, **kw).items()}
        got = _run(w.t, w.x, w.lags, world, s=w.s, y=w.y, **kw)
        if kw["kernel"] == "rectangle":
            assert np.array_equal(got["count"], ref["count"]), world
        assert np.max(np.abs(got["c"] - ref["c"])) < tol, (kw, world)


@pytest.mark.parametrize("world", [2, 5])
def test_split_long_acf(world):
    w = synth.light_curves(B=1, K=256, sizes=[1_500_000], seed=synth.BASE_SEED + 77)
    for kw, tol in ((dict(kernel="rectangle", h=0.5), 1e-10),
                    (dict(kernel="gaussian", h=0.5, path="spectral", precision="fp32"), 1e-5)):
        ref = {k: v.cpu().numpy() for k, v in api.corr(w.t, w.x, w.lags, **kw).items()}
        got = _run(w.t, w.x, w.lags, world, **kw)
        if kw["kernel"] == "rectangle":
            assert np.array_equal(got["count"], ref["count"]), world
        assert np.max(np.abs(got["c"] - ref["c"])) < tol, (kw, world)


def test_series_stats_and_pooled_call_checks():
    w = synth.ar1_acf(n=5000, K=10)
    st = api.series_stats(w.t, w.x)
    assert st["n"] == 5000 and st["flags"] == 0
    assert abs(st["mean"] - w.x.mean()) < 1e-12 and abs(st["m2"] / (w.x.var() * 5000) - 1) < 1e-12
    assert st["t_first"] == w.t[0] and st["t_last"] == w.t[-1]
    pooled = {"mean_x": st["mean"], "std_x": (st["m2"] / st["n"]) ** 0.5, "n_x": st["n"]}
    a = api.corr_pooled(w.t, w.x, w.lags, pooled, kernel="rectangle", h=1.0)
    b = api.corr(w.t, w.x, w.lags, kernel="rectangle", h=1.0)
    assert np.array_equal(a["count"].cpu().numpy(), b["count"].cpu().numpy())
    assert float((a["c"] - b["c"]).abs().max()) < 1e-12
    with pytest.raises(api.NcfError):
        api.corr_pooled(w.t, w.x, w.lags, dict(pooled, std_x=0.0), kernel="rectangle", h=1.0)
