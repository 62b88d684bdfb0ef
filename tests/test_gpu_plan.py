"""Plans (ncf_plan_*): one-time analysis, then launches without host
synchronisation or allocation -- equal to the one-shot call, reusable on new
data of the same layout, capturable in a CUDA graph, and guarded on device."""
import math

import numpy as np
import pytest
import torch

from paper_2609_03866_b300 import api, synth
from tests._gpu import max_abs, to_np

pytestmark = pytest.mark.gpu

CASES = [("rectangle", "auto", "fp64"), ("gaussian", "spectral", "fp32"),
         ("gaussian", "spectral", "fp64"), ("gaussian", "windowed", "fp64")]


def _dev(a):
    return torch.as_tensor(a, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("kernel,path,prec", CASES)
def test_plan_matches_one_shot_call_and_new_data(kernel, path, prec):
    w = synth.light_curves(B=6, n_lo=300, n_hi=5000, K=33)
    t, x, lags = _dev(w.t), _dev(w.x), _dev(w.lags)
    kw = dict(kernel=kernel, h=0.5, path=path, precision=prec)
    ref = to_np(api.corr_batch(w.offs, t, x, lags, **kw))
    plan = api.Plan(w.offs, t, x, lags, **kw)
    got = to_np(plan.execute(t, x))
    assert plan.status() == 0
    tol = 1e-12 if kernel == "rectangle" else 1e-10
    assert max_abs(got["c"], ref["c"]) < tol
    if kernel == "rectangle":
        assert np.array_equal(got["count"], ref["count"])
    # new values at the same times: the plan is reusable
    x2 = _dev(np.cos(w.x) * 3.0 + 1.0)
    ref2 = to_np(api.corr_batch(w.offs, t, x2, lags, **kw))
    got2 = to_np(plan.execute(t, x2))
    assert plan.status() == 0
    assert max_abs(got2["c"], ref2["c"]) < tol


def test_plan_ccf_lag0_matches_one_shot():
    w = synth.ou_ccf(nA=3000, nB=2500, K=21)
    t, x, s, y, lags = _dev(w.t), _dev(w.x), _dev(w.s), _dev(w.y), _dev(w.lags)
    for kernel, path in (("rectangle", "auto"), ("gaussian", "spectral")):
        kw = dict(kernel=kernel, h=0.5, path=path, norm="lag0")
        ref = to_np(api.corr_batch(w.offs, t, x, lags, offs_y=w.offs_y, s=s, y=y, **kw))
        plan = api.Plan(w.offs, t, x, lags, offs_y=w.offs_y, s=s, y=y, **kw)
        got = to_np(plan.execute(t, x, s, y))
        assert plan.status() == 0
        assert max_abs(got["c"], ref["c"]) < 1e-10


def test_plan_launch_captured_in_a_cuda_graph():
    w = synth.light_curves(B=8, n_lo=300, n_hi=4000, K=24)
    t, x, lags = _dev(w.t), _dev(w.x), _dev(w.lags)
    outs = {}
    for kernel, path, prec in (("gaussian", "spectral", "fp32"), ("rectangle", "auto", "fp64")):
        plan = api.Plan(w.offs, t, x, lags, kernel=kernel, h=0.5, path=path, precision=prec)
        out = plan.execute(t, x)          # warm-up outside the capture
        torch.cuda.synchronize()
        ref = to_np(out)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                plan.execute(t, x, out=out, stream=s)
        for v in out.values():
            v.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = to_np(out)
        assert max_abs(got["c"], ref["c"]) < 1e-12
        outs[kernel] = plan


def test_plan_device_guards():
    w = synth.light_curves(B=4, n_lo=500, n_hi=3000, K=16)
    t, x, lags = _dev(w.t), _dev(w.x), _dev(w.lags)
    plan = api.Plan(w.offs, t, x, lags, kernel="gaussian", h=0.5, path="spectral", precision="fp32")
    # shifted by far more than the padded period: outside the plan's periodic domain
    r = to_np(plan.execute(t + 5000.0, x))
    assert plan.status() & 2
    assert np.all(np.isnan(r["c"]))
    # a constant series: invalid input
    r = to_np(plan.execute(t, torch.ones_like(x)))
    assert plan.status() & 8
    # valid data again: a clean launch
    r = to_np(plan.execute(t, x))
    assert plan.status() == 0 and np.all(np.isfinite(r["c"]))
    assert plan.device_bytes > 0


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A device wait that nothing satisfies ends in the timeout status bit after
    its iteration limit (no hang, no fault); the same context then computes."""
    from paper_2609_03866_b300 import api as _api
    assert _api.selftest_bounded_wait() & 1
    w = synth.ar1_acf(n=800, K=10)
    r = _api.corr(w.t, w.x, w.lags, kernel="rectangle", h=1.0)
    assert bool(torch.isfinite(r["c"]).all())
