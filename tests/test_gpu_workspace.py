"""ncf_workspace_bytes against what the library really allocates: the bound,
computed from sizes alone, is at least ncf_plan_device_bytes of a plan built on
the data, for the light-curve batch (4096 curves x 256 lags), the seasonal OU
CCF (1e5 x 8e4 points, 200 lags) and single requests of the serving mix; the
request server admits by it."""
import numpy as np
import pytest

from paper_2609_03866_b300 import api, synth

pytestmark = pytest.mark.gpu


def _span(*ts):
    lo = min(float(np.min(t)) for t in ts)
    hi = max(float(np.max(t)) for t in ts)
    return hi - lo


def _check(offs, t, x, lags, offs_y=None, s=None, y=None, **opt):
    import torch
    B = len(offs) - 1
    if s is None:
        span = max(float(t[offs[b + 1] - 1] - t[offs[b]]) for b in range(B))
    else:
        span = max(_span(t[offs[b]:offs[b + 1]], s[offs_y[b]:offs_y[b + 1]]) for b in range(B))
    bound, _ = api.workspace_bytes(int(offs[-1]), B, lags.size, span, float(np.max(np.abs(lags))),
                                   n_y=0 if s is None else int(offs_y[-1]), **opt)
    p = api.Plan(offs, t, x, lags, offs_y=offs_y, s=s, y=y, **opt)
    used = p.device_bytes
    p.close()
    torch.cuda.synchronize()
    assert 0 < used <= bound, (opt, used, bound)
    return used, bound


def test_bound_covers_plans_on_the_light_curve_batch():
    w = synth.light_curves(B=4096, K=256)
    for opt in (dict(kernel="gaussian", h=0.5, path="spectral", precision="fp32"),
                dict(kernel="rectangle", h=0.5)):
        used, bound = _check(w.offs, w.t, w.x, w.lags, **opt)
        assert bound < 1.5 * used + (64 << 20), (opt, used, bound)   # a bound, not a guess
    # FP64 Gaussian, path chosen from the data: the bound covers either choice
    _check(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=0.5, precision="fp64")


def test_bound_covers_plans_on_the_seasonal_ou_ccf():
    w = synth.ou_ccf()
    offs = np.array([0, w.t.size], dtype=np.int64)
    offs_y = np.array([0, w.s.size], dtype=np.int64)
    for opt in (dict(kernel="rectangle", h=0.5), dict(kernel="gaussian", h=0.5, precision="fp64"),
                dict(kernel="gaussian", h=0.5, precision="fp32"), dict(kernel="rectangle", h=0.5, norm="lag0")):
        _check(offs, w.t, w.x, w.lags, offs_y=offs_y, s=w.s, y=w.y, **opt)


@pytest.mark.parametrize("n,K,ccf,kernel", [(1000, 64, False, "gaussian"), (400_000, 1024, True, "rectangle"),
                                            (2_000_000, 256, False, "gaussian"), (60_000, 1024, True, "gaussian")])
def test_bound_covers_plans_on_serving_requests(n, K, ccf, kernel):
    if ccf:
        w = synth.ou_ccf(nA=n, nB=int(0.8 * n), K=K, series=77)
        offs = np.array([0, w.t.size], dtype=np.int64)
        offs_y = np.array([0, w.s.size], dtype=np.int64)
        kw = dict(offs_y=offs_y, s=w.s, y=w.y)
    else:
        w = synth.light_curves(B=1, K=K, sizes=[n], seed=synth.BASE_SEED + 77)
        offs, kw = w.offs, {}
    opt = dict(kernel=kernel, h=0.5)
    if kernel == "gaussian":
        opt.update(path="spectral", precision="fp32")
    _check(offs, w.t, w.x, w.lags, **kw, **opt)


def test_server_admits_by_the_bound():
    w = synth.light_curves(B=1, K=256, sizes=[200_000], seed=synth.BASE_SEED + 78)
    K = w.lags.size
    opt = dict(kernel="gaussian", h=0.5, path="spectral", precision="fp32")
    ws, _ = api.workspace_bytes(w.t.size, 1, K, float(w.t[-1] - w.t[0]), float(np.max(np.abs(w.lags))), **opt)
    al = lambda b: (b + 255) // 256 * 256
    need = ws + 2 * al(8 * w.t.size) + 4 * al(8 * K)   # the workspace + the request's own copies and outputs
    small = api.Server(device=0, mem_budget_bytes=need - 1, slots=1)
    with pytest.raises(api.NcfError) as e:
        small.submit(w.t, w.x, w.lags, **opt)
    assert e.value.status == api.Server.EBUSY
    small.close()
    fits = api.Server(device=0, mem_budget_bytes=need, slots=1)
    r = fits.wait(fits.submit(w.t, w.x, w.lags, **opt))
    ref = api.corr(w.t, w.x, w.lags, **opt)["c"].cpu().numpy()
    assert np.max(np.abs(r["c"] - ref)) < 1e-6   # FP32 form: the same up to summation order
    fits.close()
