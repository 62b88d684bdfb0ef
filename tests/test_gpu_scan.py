"""GPU parity of the real-space paths against the FP64 oracle.

Rectangle: pair counts bit-exact, c within 1e-10 (the fixed-point numerator
quantises standardised values to 2^-p with p >= 27, far below that).
Gaussian windowed: c within 1e-10 of the untruncated definition at R = 8,
and window counts bit-exact against the oracle's truncated sum at R = 6.
"""
import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api, synth
from tests._gpu import max_abs, to_np

pytestmark = pytest.mark.gpu
TOL = 1e-10


def gpu(*a, **k):
    return to_np(api.corr(*a, **k))


@pytest.mark.parametrize("h", [1.0, 0.37])
def test_rectangle_acf_ar1(h):
    w = synth.ar1_acf()
    ref = oracle.corr(w.t, w.x, w.lags, "rectangle", h)
    got = gpu(w.t, w.x, w.lags, kernel="rectangle", h=h)
    assert np.array_equal(got["count"], ref["count"])
    assert np.array_equal(got["b"], ref["b"])
    assert max_abs(got["c"], ref["c"]) < TOL


def test_rectangle_ccf_seasonal_ou():
    w = synth.ou_ccf(nA=6000, nB=4800, K=57)
    ref = oracle.corr(w.t, w.x, w.lags, "rectangle", 0.5, s=w.s, y=w.y, method="windowed")
    got = gpu(w.t, w.x, w.lags, kernel="rectangle", h=0.5, s=w.s, y=w.y)
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < TOL


def test_rectangle_boundary_ties_resolved_in_fp64():
    """Integer times, integer lags, integer half-width: most window bounds land
    exactly on sample times, so every comparison goes through the FP64 band."""
    rng = np.random.default_rng(5)
    t = np.sort(rng.choice(4000, 1500, replace=False)).astype(np.float64)
    x = rng.normal(size=1500)
    lags = np.arange(-20, 21, dtype=np.float64)
    for h in (1.0, 2.0, 0.5):
        ref = oracle.corr(t, x, lags, "rectangle", h)
        got = gpu(t, x, lags, kernel="rectangle", h=h)
        assert np.array_equal(got["count"], ref["count"])
        assert max_abs(got["c"], ref["c"]) < TOL
    s = t[::2] + 3.0
    ref = oracle.corr(t, x, lags, "rectangle", 1.0, s=s, y=x[::2])
    got = gpu(t, x, lags, kernel="rectangle", h=1.0, s=s, y=x[::2])
    assert np.array_equal(got["count"], ref["count"])


def test_rectangle_mjd_offsets_duplicates_and_lag_order():
    rng = np.random.default_rng(6)
    t = np.sort(60000.0 + rng.uniform(0, 300, 2500))
    t[100:110] = t[100]                          # repeated times
    x = rng.normal(size=2500)
    lags = np.concatenate([[5.0, -3.25, 0.0, 5.0], rng.uniform(-50, 50, 20)])
    ref = oracle.corr(t, x, lags, "rectangle", 0.75, method="windowed")
    got = gpu(t, x, lags, kernel="rectangle", h=0.75)
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < TOL


@pytest.mark.parametrize("acf", [True, False])
def test_rectangle_lag0_normalisation(acf):
    w = synth.ou_ccf(nA=3000, nB=2500, K=31)
    kw = {} if acf else dict(s=w.s, y=w.y)
    ref = oracle.corr(w.t, w.x, w.lags, "rectangle", 1.0, norm="lag0", method="windowed", **kw)
    got = gpu(w.t, w.x, w.lags, kernel="rectangle", h=1.0, norm="lag0", **kw)
    assert max_abs(got["c"], ref["c"]) < TOL


def test_gaussian_windowed_matches_untruncated_definition():
    w = synth.ar1_acf()
    ref = oracle.corr(w.t, w.x, w.lags, "gaussian", 1.0)
    got = gpu(w.t, w.x, w.lags, kernel="gaussian", h=1.0, path="windowed")
    assert max_abs(got["c"], ref["c"]) < TOL
    assert np.max(np.abs(got["b"] - ref["b"]) / ref["b"]) < 1e-12


def test_gaussian_windowed_very_wide_window_underflows_to_zero_weights():
    # R = 45: weights down to exp(-1012), past the exponential's cut at z = -707.7
    # (weight 0, where the oracle's exp gives at most a few subnormals)
    w = synth.ar1_acf()
    ref = oracle.corr(w.t, w.x, w.lags, "gaussian", 1.0, trunc_R=45, method="windowed")
    got = gpu(w.t, w.x, w.lags, kernel="gaussian", h=1.0, path="windowed", trunc_R=45)
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < TOL
    assert np.max(np.abs(got["b"] - ref["b"]) / ref["b"]) < 1e-12
    full = oracle.corr(w.t, w.x, w.lags, "gaussian", 1.0)
    assert max_abs(got["c"], full["c"]) < TOL


@pytest.mark.parametrize("R", [1e4, float("inf")])
def test_gaussian_windowed_untruncated_window_far_pairs_weigh_zero(R):
    """A window far wider than the series (pairs up to 2e4 h apart, z down to -2e8):
    every far pair must weigh 0, so the result equals the untruncated definition.
    With h = 0.05 d the AR(1) series spans 2e4 h."""
    w = synth.ar1_acf()
    ref = oracle.corr(w.t, w.x, w.lags, "gaussian", 0.05)
    got = gpu(w.t, w.x, w.lags, kernel="gaussian", h=0.05, path="windowed", trunc_R=R)
    assert max_abs(got["c"], ref["c"]) < TOL
    assert np.max(np.abs(got["b"] - ref["b"]) / ref["b"]) < 1e-12
    assert np.all(np.isfinite(got["c"])) and np.all(got["b"] > 0)


def test_gaussian_windowed_paper_window_counts_exact():
    w = synth.ou_ccf(nA=4000, nB=3000, K=41)
    ref = oracle.corr(w.t, w.x, w.lags, "gaussian", 0.5, s=w.s, y=w.y, trunc_R=6, method="windowed")
    got = gpu(w.t, w.x, w.lags, kernel="gaussian", h=0.5, s=w.s, y=w.y, path="windowed", trunc_R=6)
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < TOL
    refl = oracle.corr(w.t, w.x, w.lags, "gaussian", 0.5, s=w.s, y=w.y, trunc_R=6, method="windowed",
                       norm="lag0")
    gotl = gpu(w.t, w.x, w.lags, kernel="gaussian", h=0.5, s=w.s, y=w.y, path="windowed", trunc_R=6,
               norm="lag0")
    assert max_abs(gotl["c"], refl["c"]) < TOL


def test_batch_light_curves_match_series_by_series():
    w = synth.light_curves(B=12, n_lo=200, n_hi=4000, K=40)
    for kernel, path in (("rectangle", "auto"), ("gaussian", "windowed")):
        got = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel=kernel, h=0.5, path=path))
        for b in range(w.B):
            tb, xb, _, _ = w.series(b)
            ref = oracle.corr(tb, xb, w.lags, kernel, 0.5, method="windowed",
                              trunc_R=8 if kernel == "gaussian" else 0)
            if kernel == "rectangle":
                assert np.array_equal(got["count"][b], ref["count"])
            assert max_abs(got["c"][b], ref["c"]) < TOL


def test_full_size_ccf_rectangle_counts_exact():
    """Seasonal OU CCF at full size (1e5 x 8e4 points, 200 lags)."""
    w = synth.ou_ccf()
    ref = oracle.corr(w.t, w.x, w.lags, "rectangle", 0.5, s=w.s, y=w.y, method="windowed")
    got = gpu(w.t, w.x, w.lags, kernel="rectangle", h=0.5, s=w.s, y=w.y)
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < TOL
    # the injected 15-day delay is where the CCF peaks
    assert abs(w.lags[int(np.argmax(got["c"]))] - 15.0) < 1.1


@pytest.mark.parametrize("where", ["x_nan", "x_inf", "t_inf"])
def test_non_finite_values_inside_a_batch_are_rejected(where):
    """A NaN or an infinity anywhere in a batch (here in the middle of the second
    series' third statistics chunk) is found by the statistics pass and reported,
    for the batched FP32 form and for the exact rectangle scan."""
    w = synth.light_curves(B=3, n_lo=12000, n_hi=14000, K=5, seed=9)
    t, x = w.t.copy(), w.x.copy()
    i = int(w.offs[1]) + 2 * 4096 + 77
    if where == "x_nan":
        x[i] = np.nan
    elif where == "x_inf":
        x[i] = -np.inf
    else:
        t[-1] = np.inf  # still sorted
    for kw in (dict(kernel="gaussian", h=0.5, path="spectral", precision="fp32"), dict(kernel="rectangle", h=0.5)):
        with pytest.raises(api.NcfError) as e:
            api.corr_batch(w.offs, t, x, w.lags, **kw)
        assert e.value.name == "NCF_ENONFINITE", e.value.name


def test_invalid_inputs_are_rejected_before_any_launch():
    t = np.arange(10.0)
    x = np.arange(10.0) ** 2
    lags = np.arange(3.0)
    with pytest.raises(api.NcfError) as e:
        api.corr(t[::-1].copy(), x, lags, kernel="rectangle")
    assert e.value.name == "NCF_ENOTSORTED"
    bad = x.copy()
    bad[3] = np.nan
    with pytest.raises(api.NcfError) as e:
        api.corr(t, bad, lags)
    assert e.value.name == "NCF_ENONFINITE"
    with pytest.raises(api.NcfError) as e:
        api.corr(t, np.ones(10), lags)
    assert e.value.name == "NCF_EDEGENERATE"
    with pytest.raises(api.NcfError) as e:
        api.corr(t[:1], x[:1], lags)
    assert e.value.name == "NCF_EINVAL"
    with pytest.raises(api.NcfError) as e:
        api.corr(t, x, lags, h=0.0)
    assert e.value.name == "NCF_EINVAL"
    with pytest.raises(api.NcfError) as e:
        api.corr(t, x, lags, kernel="hanning", path="spectral")
    assert e.value.name == "NCF_EUNSUPPORTED"
    # a valid call still works afterwards
    r = gpu(t, x, lags, kernel="rectangle", h=0.5)
    assert r["count"].tolist() == [10, 9, 8]
