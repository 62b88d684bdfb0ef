"""The paper's own NUFFT estimators on the GPU (ncf_corr_paper, Algorithms 1-4
with the smoothing step) against the oracle of the same algorithms."""
import math

import numpy as np
import pytest

import oracle
from oracle import paper_nufft as pn
from paper_2609_03866_b300 import api
from paper_2609_03866_b300.api import NcfError

pytestmark = pytest.mark.gpu

# Tolerance.  Both sides evaluate the same trigonometric sums in FP64: the GPU's
# type-1 transform carries the ES kernel's ~1e-14 relative error, and the
# phases of mode m are rounded at about m 1e-16 of a cycle (the oracle's
# products k tau~ more coarsely than the GPU's 64-bit fixed-point phases).
# At N1 ~ 1.2e4 the estimates agree to 2e-13; the bound allows for the phase
# error growing with N1 across these cases.
C_TOL = 1e-11
B_RTOL = 1e-10


def _irregular(n, span, seed, phase=0.0):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, span, n)) + phase
    x = np.sin(t / 5.0) + 0.5 * rng.standard_normal(n)
    return t, x


def _lags(K, lo, hi, seed):
    rng = np.random.default_rng(seed)
    lags = rng.uniform(lo, hi, K)
    lags[3] = 0.0            # a requested zero lag beside the prepended one
    lags[7] = lags[11]       # a repeated lag
    return lags


def _run(t, x, lags, kernel, h, s=None, y=None, N1=0):
    r = api.corr_paper(t, x, lags, kernel=kernel, h=h, s=s, y=y, N1=N1)
    return r["c"].cpu().numpy(), r["b"].cpu().numpy()


@pytest.mark.parametrize("kernel,h", [("gaussian", 0.7), ("rectangle", 1.2), ("rectangle", 1.5)])
def test_acf_matches_oracle(kernel, h):
    t, x = _irregular(300, 150.0, 1)
    lags = _lags(37, -20.0, 25.0, 2)
    c, b = _run(t, x, lags, kernel, h)
    ref = pn.acf(t, x, lags, kernel, h)
    print("acf", kernel, h, ref["N1"], np.abs(c - ref["c"]).max(), np.abs(b / ref["b"] - 1).max())
    np.testing.assert_allclose(c, ref["c"], rtol=0, atol=C_TOL)
    np.testing.assert_allclose(b, ref["b"], rtol=B_RTOL)


@pytest.mark.parametrize("kernel,h", [("gaussian", 0.7), ("rectangle", 1.5)])
def test_ccf_matches_oracle(kernel, h):
    t, x = _irregular(260, 140.0, 3)
    s, y = _irregular(210, 120.0, 4, phase=9.0)
    lags = _lags(37, -30.0, 30.0, 5)
    c, b = _run(t, x, lags, kernel, h, s=s, y=y)
    ref = pn.ccf(t, x, s, y, lags, kernel, h)
    print("ccf", kernel, h, ref["N1"], np.abs(c - ref["c"]).max(), np.abs(b / ref["b"] - 1).max())
    np.testing.assert_allclose(c, ref["c"], rtol=0, atol=C_TOL)
    np.testing.assert_allclose(b, ref["b"], rtol=B_RTOL)


@pytest.mark.parametrize("kernel,h", [("gaussian", 0.7), ("rectangle", 1.5)])
def test_long_lag_arrays_through_the_type2_transform(kernel, h):
    # from 48 evaluation lags on, the raw correlation comes from a type-2 transform
    # (deconvolution, one FFT, 16-tap interpolation) instead of the direct mode sum
    t, x = _irregular(280, 140.0, 12)
    s, y = _irregular(230, 130.0, 13, phase=6.0)
    lags = _lags(120, -35.0, 35.0, 14)
    c, b = _run(t, x, lags, kernel, h, s=s, y=y)
    ref = pn.ccf(t, x, s, y, lags, kernel, h)
    print("type2 ccf", kernel, h, ref["N1"], np.abs(c - ref["c"]).max())
    np.testing.assert_allclose(c, ref["c"], rtol=0, atol=C_TOL)
    np.testing.assert_allclose(b, ref["b"], rtol=B_RTOL)
    c, b = _run(t, x, lags, kernel, h)
    ref = pn.acf(t, x, lags, kernel, h)
    np.testing.assert_allclose(c, ref["c"], rtol=0, atol=C_TOL)


@pytest.mark.parametrize("N1", [4096, 4097])
def test_explicit_grid_sizes(N1):
    # even N1 carries the unpaired mode -N1/2 with weight 1
    t, x = _irregular(180, 90.0, 6)
    s, y = _irregular(150, 80.0, 7, phase=4.0)
    lags = _lags(20, -10.0, 15.0, 8)
    c, _ = _run(t, x, lags, "gaussian", 1.0, s=s, y=y, N1=N1)
    ref = pn.ccf(t, x, s, y, lags, "gaussian", 1.0, N1=N1)
    np.testing.assert_allclose(c, ref["c"], rtol=0, atol=C_TOL)
    c, _ = _run(t, x, lags, "rectangle", 1.5, N1=N1)
    ref = pn.acf(t, x, lags, "rectangle", 1.5, N1=N1)
    np.testing.assert_allclose(c, ref["c"], rtol=0, atol=C_TOL)


@pytest.mark.parametrize("kernel,h", [("gaussian", 1.0), ("rectangle", 1.5)])
def test_integer_days_with_N1_a_multiple_of_L_give_the_kernel_estimator(kernel, h):
    # the exact reduction of the pins, at ten thousand points: every nonzero
    # integer separation falls on a zero of the Dirichlet kernel
    rng = np.random.default_rng(9)
    n = 12000
    t = np.arange(n, dtype=np.float64)
    t = t[rng.uniform(size=n) > 0.2]
    v = np.zeros(t.size)
    for i in range(1, t.size):
        v[i] = 0.9 * v[i - 1] + rng.standard_normal()
    lags = np.concatenate([np.arange(-30.0, 0.0), np.arange(1.0, 31.0)])
    span = t[-1] - t[0]
    N1 = int(math.ceil(32 * t.size / span)) * int(span + 60.0)   # a multiple of L = span + 2 max|tau|
    c, b = _run(t, v, lags, kernel, h, N1=N1)
    ex = oracle.corr(t, v, lags, kernel, h, norm="lag0", method="windowed", trunc_R=6.0)
    r = int(4 * h + 0.5) if kernel == "gaussian" else pn.box_size(h) // 2
    inner = np.abs(lags) <= 30 - r - 1
    np.testing.assert_allclose(c[inner], ex["c"][inner], rtol=0, atol=1e-5 if kernel == "gaussian" else 1e-10)
    np.testing.assert_allclose(b, np.maximum(ex["b"], 1e-16), rtol=B_RTOL)


def test_acf_equals_ccf_of_itself_at_a_large_size():
    # Algorithms 3 and 4 meet on the symmetric lag array (the identity of the pins)
    t, x = _irregular(60000, 30000.0, 10)
    h = 0.8
    n_h = max(math.ceil(4 * h) + 2, 5)
    lags = np.concatenate([np.arange(-n_h, 0.0), np.arange(1.0, n_h + 1)])
    a, _ = _run(t, x, lags, "gaussian", h)
    c, _ = _run(t, x, lags, "gaussian", h, s=t, y=x)
    np.testing.assert_allclose(a, c, rtol=0, atol=1e-9)
    np.testing.assert_allclose(a, a[::-1], rtol=0, atol=1e-9)


def test_error_statuses():
    t, x = _irregular(50, 20.0, 11)
    lags = np.array([1.0, 2.0])
    with pytest.raises(NcfError) as e:
        api.corr_paper(t, x, lags, kernel="hanning", h=1.0)
    assert e.value.name == "NCF_EUNSUPPORTED"
    with pytest.raises(NcfError) as e:
        api.corr_paper(t, x, lags, kernel="rectangle", h=0.2)   # round(0.4) = 0 entries
    assert e.value.name == "NCF_EINVAL"
    with pytest.raises(NcfError) as e:
        api.corr_paper(t, x, lags, kernel="gaussian", h=1.0, N1=1 << 27)
    assert e.value.name == "NCF_EUNSUPPORTED"
    with pytest.raises(NcfError) as e:
        api.corr_paper(np.full(50, 3.0), x, lags, kernel="gaussian", h=1.0)
    assert e.value.name == "NCF_EDEGENERATE"
