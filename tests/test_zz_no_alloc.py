"""The allocation-free entry point ncf_corr_window_static, called through the
C ABI, against the regular ncf_corr (Gaussian, windowed path).

It serves callers that may not allocate device memory while running; its
scratch is one fixed array shared by every call, so the test makes several
calls in a row (the second and third must not see the first one's sums).
Kept in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_2609_03866_b300 import api, synth

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _prepared(t, x, lags, h, s=None, y=None, trunc_R=0.0):
    """Device copies of the inputs and outputs, then a closure that makes one call
    of the entry point through the C ABI (nothing else) and returns its status."""
    import torch
    L = api.lib()
    fn = L.ncf_corr_window_static
    vp = ctypes.c_void_p
    fn.argtypes = [vp, vp, ctypes.c_int64, vp, vp, ctypes.c_int64, vp, ctypes.c_int64,
                   ctypes.c_double, ctypes.c_double, vp, vp, vp]
    fn.restype = ctypes.c_int
    dev = torch.device("cuda", 0)
    T = torch.as_tensor(t, dtype=torch.float64, device=dev)
    X = torch.as_tensor(x, dtype=torch.float64, device=dev)
    Lg = torch.as_tensor(lags, dtype=torch.float64, device=dev)
    S = torch.as_tensor(s, dtype=torch.float64, device=dev) if s is not None else None
    Y = torch.as_tensor(y, dtype=torch.float64, device=dev) if y is not None else None
    c = torch.empty(Lg.numel(), dtype=torch.float64, device=dev)
    b = torch.empty_like(c)
    stream = vp(torch.cuda.current_stream(dev).cuda_stream)
    p = lambda a: vp(a.data_ptr()) if a is not None else vp(0)
    keep = (T, X, Lg, S, Y)

    def call():
        _ = keep
        return fn(p(T), p(X), T.numel(), p(S), p(Y), 0 if S is None else S.numel(), p(Lg), Lg.numel(),
                  float(h), float(trunc_R), p(c), p(b), stream)

    return call, c, b


def _static(t, x, lags, h, s=None, y=None, trunc_R=0.0):
    import torch
    call, c, b = _prepared(t, x, lags, h, s=s, y=y, trunc_R=trunc_R)
    rc = call()
    torch.cuda.synchronize()
    return rc, c.cpu().numpy(), b.cpu().numpy()


def _regular(t, x, lags, h, s=None, y=None, trunc_R=0.0):
    r = api.corr(t, x, lags, kernel="gaussian", h=h, s=s, y=y, path="windowed", trunc_R=trunc_R)
    return r["c"].cpu().numpy(), r["b"].cpu().numpy()


def test_static_scratch_entry_point_matches_ncf_corr():
    a = synth.ar1_acf(n=3000, K=40)
    c = synth.ou_ccf(nA=5000, nB=4000, K=33)
    ref_a = _regular(a.t, a.x, a.lags, 1.0)
    ref_c = _regular(c.t, c.x, c.lags, 0.5, s=c.s, y=c.y, trunc_R=6)
    for _ in range(2):   # two rounds of calls on the same shared scratch
        rc, ca, ba = _static(a.t, a.x, a.lags, 1.0)
        assert rc == 0
        assert np.max(np.abs(ca - ref_a[0])) < TOL
        assert np.max(np.abs(ba / ref_a[1] - 1)) < 1e-12
        rc, cc, _ = _static(c.t, c.x, c.lags, 0.5, s=c.s, y=c.y, trunc_R=6)
        assert rc == 0
        assert np.max(np.abs(cc - ref_c[0])) < TOL


def test_static_scratch_rejects_sizes_beyond_its_limit():
    t = np.arange(300000, dtype=np.float64)
    x = np.sin(t)
    rc, _, _ = _static(t, x, np.array([0.0, 1.0]), 1.0)
    assert rc == 9   # NCF_EUNSUPPORTED
    rc, _, _ = _static(t[:100], x[:100], np.arange(1025, dtype=np.float64), 1.0)
    assert rc == 9


def test_static_scratch_allocates_no_device_memory():
    """After the first call (which looks up the scratch address), repeated calls
    leave the device's free memory unchanged: nothing is allocated or freed."""
    import torch
    a = synth.ar1_acf(n=3000, K=40)
    call, c, _ = _prepared(a.t, a.x, a.lags, 1.0)
    assert call() == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    for _ in range(5):
        assert call() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0, (free0, free1)
    ref = _regular(a.t, a.x, a.lags, 1.0)
    assert np.max(np.abs(c.cpu().numpy() - ref[0])) < TOL


def test_static_scratch_at_its_size_limits():
    """Exactly the largest series (262144 points) and lag count (1024) the fixed
    scratch holds, twice in a row, against ncf_corr.  A sparse series (one point
    per 10 days on average) keeps the window's pairs few."""
    rng = np.random.default_rng(44)
    n, K = 262144, 1024
    t = np.sort(rng.uniform(0.0, 10.0 * n, n))
    x = rng.normal(size=n) + np.sin(t / 37.0)
    lags = np.linspace(0.0, 2000.0, K)
    ref = _regular(t, x, lags, 4.0)
    for _ in range(2):
        rc, c, b = _static(t, x, lags, 4.0)
        assert rc == 0
        assert np.max(np.abs(c - ref[0])) < TOL
        assert np.max(np.abs(b / ref[1] - 1)) < 1e-12
