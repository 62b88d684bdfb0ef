"""Plans of several estimators (ncf_plan_create_multi): one statistics pass per
execution, every option set's result equal to its own plan's, capturable in a
CUDA graph (the benchmark's step), and the shared status word reports a guard
raised by any set."""
import numpy as np
import pytest
import torch

from paper_2609_03866_b300 import api, synth
from tests._gpu import to_np

pytestmark = pytest.mark.gpu
OPTS = [dict(kernel="gaussian", h=0.5, path="spectral", precision="fp32"), dict(kernel="rectangle", h=0.5),
        dict(kernel="gaussian", h=0.5, path="spectral", precision="fp64", norm="lag0")]


def _dev(a):
    return torch.as_tensor(a, dtype=torch.float64, device="cuda")


def test_multi_plan_equals_single_plans_and_replays_in_a_graph():
    w = synth.light_curves(B=24, n_lo=300, n_hi=20_000, K=40, seed=synth.BASE_SEED + 71)
    t, x, lags = _dev(w.t), _dev(w.x), _dev(w.lags)
    mp = api.MultiPlan(w.offs, t, x, lags, OPTS)
    outs = mp.execute(t, x)
    assert mp.status() == 0
    got = [to_np(o) for o in outs]
    for o, g in zip(OPTS, got):
        ref = to_np(api.Plan(w.offs, t, x, lags, **o).execute(t, x))
        if o["kernel"] == "rectangle":
            assert np.array_equal(g["count"], ref["count"]) and np.array_equal(g["c"], ref["c"])
        else:
            assert np.max(np.abs(g["c"] - ref["c"])) < (1e-6 if o["precision"] == "fp32" else 1e-12)
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            mp.execute(t, x, outs=outs, stream=s)
    for o in outs:
        for v in o.values():
            v.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for o, g in zip(outs, got):
        assert np.max(np.abs(o["c"].cpu().numpy() - g["c"])) < 1e-6
    # new data of the same layout: the guard of the statistics pass covers every set
    x_bad = x.clone()
    x_bad[int(w.offs[3]):int(w.offs[4])] = 1.0       # a constant series
    mp.execute(t, x_bad, outs=outs)
    assert mp.status() != 0
    assert torch.isnan(outs[1]["c"]).all() and torch.isnan(outs[0]["c"]).all()
    mp.close()
