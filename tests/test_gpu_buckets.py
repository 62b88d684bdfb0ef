"""Per-series grid sizing: a batch whose series span very different times is
split into buckets of series needing the same grid size, each evaluated on its
own period and grid (Algorithm 1 per bucket), with every series' result in its
own output row.

The split must give the same estimates as one common grid (the spectral path's
accuracy does not depend on the period once it covers span + max lag + the
alias margin): FP64 within 1e-10 of the one-grid result and of the oracle, the
FP32 form within 1e-5 of FP64, for ACF and CCF batches, one-shot calls and
plans replayed from a CUDA graph.  A split plan needs no more device memory
than ncf_workspace_bytes' size-only bound.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api
from tests._gpu import to_np

pytestmark = pytest.mark.gpu


def _one_grid(fn):
    old = os.environ.get("NCF_SPEC_BUCKETS")
    os.environ["NCF_SPEC_BUCKETS"] = "0"
    try:
        return fn()
    finally:
        if old is None:
            os.environ.pop("NCF_SPEC_BUCKETS", None)
        else:
            os.environ["NCF_SPEC_BUCKETS"] = old


def _mixed_spans(B=60, seed=3, n_lo=400, n_hi=3000):
    """Series of spans from 20 d to 1400 d (log-uniform), uniform times, an AR-like
    signal plus noise; deliberately in no particular order of span."""
    rng = np.random.default_rng(seed)
    spans = np.exp(rng.uniform(np.log(20.0), np.log(1400.0), B))
    ts, xs = [], []
    for b in range(B):
        n = int(rng.integers(n_lo, n_hi))
        t = np.sort(rng.uniform(0.0, spans[b], n)) + rng.uniform(0, 5000)
        x = np.sin(2 * np.pi * t / rng.uniform(2, 40)) + rng.normal(size=n)
        ts.append(t)
        xs.append(x)
    offs = np.concatenate([[0], np.cumsum([t.size for t in ts])]).astype(np.int64)
    return offs, np.concatenate(ts), np.concatenate(xs), spans


def test_fp64_acf_split_matches_one_grid_and_oracle():
    offs, t, x, _ = _mixed_spans()
    lags = np.linspace(0.0, 15.0, 33)
    ctx = api.Context()
    try:
        split = to_np(api.corr_batch(offs, t, x, lags, kernel="gaussian", h=0.5, path="spectral", ctx=ctx))
        assert ctx.last_plan()["buckets"] > 1
        one = _one_grid(lambda: to_np(api.corr_batch(offs, t, x, lags, kernel="gaussian", h=0.5,
                                                     path="spectral", ctx=ctx)))
        assert ctx.last_plan()["buckets"] == 1
    finally:
        ctx.close()
    assert np.max(np.abs(split["c"] - one["c"])) < 1e-10
    assert np.max(np.abs(split["b"] / one["b"] - 1.0)) < 1e-10
    for b in (0, 7, 23, 41, 59):
        tb, xb = t[offs[b]:offs[b + 1]], x[offs[b]:offs[b + 1]]
        ref = oracle.corr(tb, xb, lags, "gaussian", 0.5, method="windowed", trunc_R=8.0)
        assert np.max(np.abs(split["c"][b] - ref["c"])) < 1e-10, b


def test_fp32_acf_split_matches_fp64():
    # a split pays for its per-bucket tables (128-series tensor-core tiles, lag
    # tables) only on batches of some size: 300 series here
    offs, t, x, _ = _mixed_spans(B=300, seed=4, n_lo=800, n_hi=2500)
    lags = np.linspace(0.0, 15.0, 33)
    ctx = api.Context()
    try:
        f32 = to_np(api.corr_batch(offs, t, x, lags, kernel="gaussian", h=0.5, path="spectral",
                                   precision="fp32", ctx=ctx))
        assert ctx.last_plan()["buckets"] > 1
    finally:
        ctx.close()
    f64 = _one_grid(lambda: to_np(api.corr_batch(offs, t, x, lags, kernel="gaussian", h=0.5, path="spectral")))
    assert np.max(np.abs(f32["c"] - f64["c"])) < 1e-5


def test_fp64_ccf_split_matches_one_grid():
    offs, t, x, spans = _mixed_spans(B=30, seed=5)
    rng = np.random.default_rng(6)
    # y: a delayed noisy copy sampled at its own times over the same span
    ss, ys = [], []
    for b in range(30):
        tb, xb = t[offs[b]:offs[b + 1]], x[offs[b]:offs[b + 1]]
        sb = np.sort(rng.uniform(tb[0], tb[-1], max(50, tb.size // 2)))
        ss.append(sb)
        ys.append(np.interp(sb - 1.5, tb, xb) + 0.3 * rng.normal(size=sb.size))
    oy = np.concatenate([[0], np.cumsum([s.size for s in ss])]).astype(np.int64)
    s, y = np.concatenate(ss), np.concatenate(ys)
    lags = np.linspace(-10.0, 10.0, 41)
    kw = dict(kernel="gaussian", h=0.5, offs_y=oy, s=s, y=y, path="spectral")
    ctx = api.Context()
    try:
        split = to_np(api.corr_batch(offs, t, x, lags, ctx=ctx, **kw))
        assert ctx.last_plan()["buckets"] > 1
    finally:
        ctx.close()
    one = _one_grid(lambda: to_np(api.corr_batch(offs, t, x, lags, **kw)))
    assert np.max(np.abs(split["c"] - one["c"])) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_split_plan_in_a_cuda_graph_and_within_the_memory_bound(precision):
    import torch
    B = 300
    offs, t, x, spans = _mixed_spans(B=B, seed=8, n_lo=800, n_hi=2000)
    lags = np.linspace(0.0, 15.0, 17)
    dev = torch.device("cuda", 0)
    T, X, Lg = (torch.as_tensor(a, device=dev) for a in (t, x, lags))
    ref = to_np(api.corr_batch(offs, T, X, Lg, kernel="gaussian", h=0.5, path="spectral", precision=precision))
    plan = api.Plan(offs, T, X, Lg, kernel="gaussian", h=0.5, path="spectral", precision=precision)
    assert plan.ctx.last_plan()["buckets"] > 1
    out = plan.execute(T, X)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            plan.execute(T, X, out=out, stream=st)
    for v in out.values():
        v.zero_()
    g.replay()
    torch.cuda.synchronize()
    got = to_np(out)
    assert plan.status() == 0
    # FP32 spreading adds with atomics in no fixed order: runs differ in the last
    # FP32 bits; FP64 runs agree to rounding
    assert np.max(np.abs(got["c"] - ref["c"])) < (1e-12 if precision == "fp64" else 1e-6)
    span = float(max(t[offs[b + 1] - 1] - t[offs[b]] for b in range(B)))
    bound, _ = api.workspace_bytes(t.size, B, lags.size, span, float(lags.max()), kernel="gaussian", h=0.5,
                                   path="spectral", precision=precision)
    assert plan.device_bytes <= bound


def _three_spans(seed=11):
    """Three series of very different spans (20, 200, 1400 d): one series per grid
    size, so each bucket holds a single series and sums its modes directly."""
    rng = np.random.default_rng(seed)
    ts, xs = [], []
    for span, n in ((20.0, 3000), (200.0, 5000), (1400.0, 8000)):
        t = np.sort(rng.uniform(0.0, span, n)) + 100.0
        ts.append(t)
        xs.append(np.sin(2 * np.pi * t / 3.7) + rng.normal(size=n))
    offs = np.concatenate([[0], np.cumsum([t.size for t in ts])]).astype(np.int64)
    return offs, np.concatenate(ts), np.concatenate(xs)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("norm", ["none", "lag0"])
def test_single_series_buckets_and_pearson(precision, tol, norm):
    offs, t, x = _three_spans()
    lags = np.linspace(0.0, 8.0, 25)
    ctx = api.Context()
    try:
        split = to_np(api.corr_batch(offs, t, x, lags, kernel="gaussian", h=0.5, path="spectral",
                                     precision=precision, norm=norm, ctx=ctx))
        assert ctx.last_plan()["buckets"] == 3
    finally:
        ctx.close()
    one = _one_grid(lambda: to_np(api.corr_batch(offs, t, x, lags, kernel="gaussian", h=0.5, path="spectral",
                                                 precision="fp64", norm=norm)))
    assert np.max(np.abs(split["c"] - one["c"])) < tol
    for b in range(3):
        tb, xb = t[offs[b]:offs[b + 1]], x[offs[b]:offs[b + 1]]
        ref = oracle.corr(tb, xb, lags, "gaussian", 0.5, norm=norm, method="windowed", trunc_R=8.0)
        assert np.max(np.abs(split["c"][b] - ref["c"])) < tol, b


def test_ccf_buckets_with_pearson():
    offs, t, x, _ = _mixed_spans(B=24, seed=12, n_lo=600, n_hi=2000)
    rng = np.random.default_rng(13)
    ss, ys = [], []
    for b in range(24):
        tb, xb = t[offs[b]:offs[b + 1]], x[offs[b]:offs[b + 1]]
        sb = np.sort(rng.uniform(tb[0], tb[-1], tb.size))
        ss.append(sb)
        ys.append(np.interp(sb - 0.7, tb, xb) + 0.5 * rng.normal(size=sb.size))
    oy = np.concatenate([[0], np.cumsum([s.size for s in ss])]).astype(np.int64)
    s, y = np.concatenate(ss), np.concatenate(ys)
    lags = np.linspace(-6.0, 6.0, 25)
    kw = dict(kernel="gaussian", h=0.5, offs_y=oy, s=s, y=y, path="spectral", norm="lag0")
    ctx = api.Context()
    try:
        split = to_np(api.corr_batch(offs, t, x, lags, ctx=ctx, **kw))
        assert ctx.last_plan()["buckets"] > 1
    finally:
        ctx.close()
    one = _one_grid(lambda: to_np(api.corr_batch(offs, t, x, lags, **kw)))
    assert np.max(np.abs(split["c"] - one["c"])) < 1e-10
    b = 5
    ref = oracle.corr(t[offs[b]:offs[b + 1]], x[offs[b]:offs[b + 1]], lags, "gaussian", 0.5,
                      s=s[oy[b]:oy[b + 1]], y=y[oy[b]:oy[b + 1]], norm="lag0", method="windowed", trunc_R=8.0)
    assert np.max(np.abs(split["c"][b] - ref["c"])) < 1e-10
