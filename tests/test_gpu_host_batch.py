"""The host-buffer batch call (ncf_corr_batch_host): large batches are evaluated
as chunks of series whose uploads overlap the previous chunk's evaluation; the
results equal the device-buffer call on the same data (rectangle exactly; the
Gaussian within its tolerance, since each chunk takes its own spectral period)."""
import numpy as np
import pytest
import torch

from paper_2609_03866_b300 import api, synth
from tests._gpu import max_abs, to_np

pytestmark = pytest.mark.gpu


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


def host_call(w, **kw):
    B, K = w.B, w.lags.size
    out = {"c": torch.empty(B, K, dtype=torch.float64).pin_memory(),
           "b": torch.empty(B, K, dtype=torch.float64).pin_memory(),
           "count": torch.empty(B, K, dtype=torch.int64).pin_memory()}
    api.corr_batch_host(w.offs, pinned(w.t), pinned(w.x), pinned(w.lags), out=out, **kw)
    return {k: v.numpy() for k, v in out.items()}


def test_chunked_host_batch_equals_device_batch():
    w = synth.light_curves(B=700, n_lo=20_000, n_hi=200_000, K=64, seed=synth.BASE_SEED + 77)
    assert w.t.size * 16 > (256 << 20)          # large enough for the chunked path
    for kw, tol in [(dict(kernel="rectangle", h=0.5), 0.0),
                    (dict(kernel="gaussian", h=0.5, path="spectral", precision="fp64"), 1e-10),
                    (dict(kernel="gaussian", h=0.5, path="spectral", precision="fp32"), 1e-5)]:
        got = host_call(w, **kw)
        ref = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, **kw))
        if kw["kernel"] == "rectangle":
            assert np.array_equal(got["count"], ref["count"])
            assert np.array_equal(got["c"], ref["c"])
        else:
            assert max_abs(got["c"], ref["c"]) <= tol


def test_small_host_batch_ccf_and_pearson():
    w = synth.light_curves(B=5, n_lo=500, n_hi=3000, K=21, seed=synth.BASE_SEED + 78)
    c = synth.ou_ccf(nA=3000, nB=2400, K=17)
    got = host_call(w, kernel="rectangle", h=0.5, norm="lag0")
    ref = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="rectangle", h=0.5, norm="lag0"))
    assert np.array_equal(got["count"], ref["count"]) and np.array_equal(got["c"], ref["c"])
    out = {"c": torch.empty(1, c.lags.size, dtype=torch.float64).pin_memory()}
    api.corr_batch_host(c.offs, pinned(c.t), pinned(c.x), pinned(c.lags), kernel="gaussian", h=0.5,
                        offs_y=c.offs_y, s=pinned(c.s), y=pinned(c.y), out=out)
    ref = to_np(api.corr(c.t, c.x, c.lags, kernel="gaussian", h=0.5, s=c.s, y=c.y))
    assert max_abs(out["c"].numpy()[0], ref["c"]) < 1e-10


def test_several_estimators_from_one_upload_equal_separate_calls():
    # ncf_corr_batch_host_multi: the same chunks (and spectral periods) as the
    # single call, so each option set matches its own host call: the rectangle
    # exactly, the Gaussian up to the order of the spreading's atomic additions
    w = synth.light_curves(B=700, n_lo=20_000, n_hi=200_000, K=64, seed=synth.BASE_SEED + 77)
    opts = [dict(kernel="gaussian", h=0.5, path="spectral", precision="fp32"),
            dict(kernel="rectangle", h=0.5),
            dict(kernel="gaussian", h=0.5, path="spectral", precision="fp64", norm="lag0")]
    tols = [1e-6, 0.0, 1e-12]
    outs = api.corr_batch_host_multi(w.offs, pinned(w.t), pinned(w.x), pinned(w.lags), opts)
    for o, tol, got in zip(opts, tols, outs):
        ref = host_call(w, **o)
        if tol == 0.0:
            for key in ("c", "b", "count"):
                assert np.array_equal(got[key].numpy(), ref[key]), (o, key)
        else:
            assert max_abs(got["c"].numpy(), ref["c"]) <= tol, o
            assert np.allclose(got["b"].numpy(), ref["b"], rtol=10 * tol, atol=0), o


def test_several_estimators_ccf_with_optional_outputs_left_out():
    c = synth.ou_ccf(nA=3000, nB=2400, K=17)
    opts = [dict(kernel="rectangle", h=0.5), dict(kernel="gaussian", h=0.5, path="windowed", trunc_R=8.0)]
    outs = [{"c": torch.empty(1, c.lags.size, dtype=torch.float64)},
            {"c": torch.empty(1, c.lags.size, dtype=torch.float64),
             "count": torch.empty(1, c.lags.size, dtype=torch.int64)}]
    api.corr_batch_host_multi(c.offs, c.t, c.x, c.lags, opts, offs_y=c.offs_y, s=c.s, y=c.y, outs=outs)
    for o, got in zip(opts, outs):
        ref = to_np(api.corr(c.t, c.x, c.lags, s=c.s, y=c.y, **o))
        assert max_abs(got["c"].numpy()[0], ref["c"]) < 1e-10
        if "count" in got:
            assert np.array_equal(got["count"].numpy()[0], ref["count"])


def test_chunked_host_batch_ccf_and_repeated_calls():
    """A chunked batch of cross-correlations (both sides uploaded per chunk, each
    chunk's statistics stage beside the previous chunk's evaluation), called
    twice on one context with a device-buffer call in between: every call equals
    the device-buffer call (the rectangle exactly; the Gaussian through the FP64
    and FP32 spectral forms within their tolerances)."""
    rng = np.random.default_rng(31)
    xs, ys = [], []
    for b in range(24):
        c = synth.ou_ccf(nA=int(rng.integers(350_000, 450_000)), nB=int(rng.integers(350_000, 450_000)), K=33,
                         seed=500 + b)
        xs.append((c.t, c.x))
        ys.append((c.s, c.y))
        lags = c.lags
    ox = np.concatenate([[0], np.cumsum([t.size for t, _ in xs])]).astype(np.int64)
    oy = np.concatenate([[0], np.cumsum([s.size for s, _ in ys])]).astype(np.int64)
    t = np.concatenate([a for a, _ in xs]); x = np.concatenate([b for _, b in xs])
    s = np.concatenate([a for a, _ in ys]); y = np.concatenate([b for _, b in ys])
    assert (t.size + s.size) * 16 > (256 << 20)  # the chunked path
    kw = dict(kernel="rectangle", h=0.5, offs_y=oy)
    ctx = api.Context()
    try:
        ref = to_np(api.corr_batch(ox, t, x, lags, s=s, y=y, ctx=ctx, **kw))
        for _ in range(2):
            B, K = ox.size - 1, lags.size
            out = {"c": torch.empty(B, K, dtype=torch.float64).pin_memory(),
                   "count": torch.empty(B, K, dtype=torch.int64).pin_memory()}
            api.corr_batch_host(ox, pinned(t), pinned(x), pinned(lags), s=pinned(s), y=pinned(y), out=out, ctx=ctx,
                                **kw)
            assert np.array_equal(out["count"].numpy(), ref["count"])
            assert np.array_equal(out["c"].numpy(), ref["c"])
            dev = to_np(api.corr_batch(ox, t, x, lags, s=s, y=y, ctx=ctx, **kw))
            assert np.array_equal(dev["c"], ref["c"])
        # the Gaussian through both spectral forms (each chunk on its own period)
        for gk, tol in [(dict(path="spectral", precision="fp64"), 1e-10),
                        (dict(path="spectral", precision="fp32"), 1e-5)]:
            g = dict(kernel="gaussian", h=0.5, offs_y=oy, **gk)
            gref = to_np(api.corr_batch(ox, t, x, lags, s=s, y=y, ctx=ctx, **g))
            out = {"c": torch.empty(ox.size - 1, lags.size, dtype=torch.float64).pin_memory()}
            api.corr_batch_host(ox, pinned(t), pinned(x), pinned(lags), s=pinned(s), y=pinned(y), out=out, ctx=ctx,
                                **g)
            assert max_abs(out["c"].numpy(), gref["c"]) <= tol
    finally:
        ctx.close()


def test_rectangle_result_of_a_series_does_not_depend_on_its_batch():
    """The rectangle's fixed-point values are scaled by each series' own length
    (value_bits), so a series gives the same bits alone and in a batch beside a
    series 30 times longer (whose length alone sets a coarser scale)."""
    small = synth.light_curves(B=1, K=40, sizes=[3000], seed=synth.BASE_SEED + 301)
    big = synth.light_curves(B=1, K=40, sizes=[90_000], seed=synth.BASE_SEED + 302)
    lags = small.lags
    alone = to_np(api.corr_batch(small.offs, small.t, small.x, lags, kernel="rectangle", h=0.5))
    offs = np.array([0, small.t.size, small.t.size + big.t.size], dtype=np.int64)
    t = np.concatenate([small.t, big.t]); x = np.concatenate([small.x, big.x])
    both = to_np(api.corr_batch(offs, t, x, lags, kernel="rectangle", h=0.5))
    assert np.array_equal(both["count"][0], alone["count"][0])
    assert np.array_equal(both["c"][0], alone["c"][0])
