"""Pins for the FP64 CPU oracle against facts fixed by the paper and by the
mathematics -- never against the oracle itself.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
sign or index error, a transposed operand, a wrong constant or width) fails
at least one of them:

* exhaustive enumeration in exact rationals (rectangle) and 50-digit
  arithmetic (Gaussian) on a dozen points, including pairs that sit exactly on
  the closed window boundaries of Algorithm 6;
* the textbook regular-grid estimator, Eq. acf_regular (via numpy.correlate);
* moments of the Gaussian effective pair count over the lag axis (kernel
  normalisation, centre and width of Eq. Gaussian_kernel);
* rectangle windows tiling the lag axis count every pair exactly once;
* symmetries stated in the appendix: C_yx(tau) = C_xy(-tau), CCF of a series
  with itself equals its ACF, ACF evenness; invariance under affine rescaling;
* a copy shifted by tau0 peaks at +tau0 with count n and c = 1 (Sec. 3.1);
* the windowed scan (Algorithms 5-8) against the direct double sum.
"""
import numpy as np
import pytest

import oracle


def _rng(seed):
    return np.random.default_rng(seed)


def _dyadic_series(rng, n, span_eighths=96):
    t = np.sort(rng.choice(span_eighths, size=n, replace=False)).astype(np.float64) / 8.0
    x = rng.integers(-8, 9, size=n).astype(np.float64) / 4.0
    x[0] += 3.0  # guarantee nonzero variance
    return t, x


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("h", [0.5, 1.0, 1.25])
def test_rectangle_direct_matches_exact_enumeration_acf(seed, h):
    rng = _rng(seed)
    t, x = _dyadic_series(rng, 11)
    lags = np.arange(0, 41, dtype=np.float64) / 8.0  # lags land exactly on pair separations
    cnt, nums, cs = oracle.exact_rectangle(t, x, lags, h)
    r = oracle.corr(t, x, lags, "rectangle", h)
    assert r["count"].tolist() == cnt
    assert np.max(np.abs(r["num"] - np.array([float(v) for v in nums]))) < 1e-13
    assert np.max(np.abs(r["c"] - np.array([float(v) for v in cs]))) < 1e-14
    assert np.array_equal(r["b"], np.array(cnt, dtype=np.float64))


@pytest.mark.parametrize("seed", [4, 5])
@pytest.mark.parametrize("h", [0.5, 0.875])
def test_rectangle_direct_matches_exact_enumeration_ccf(seed, h):
    rng = _rng(seed)
    t, x = _dyadic_series(rng, 10)
    s, y = _dyadic_series(rng, 12)
    lags = np.arange(-40, 41, dtype=np.float64) / 8.0
    cnt, nums, cs = oracle.exact_rectangle(t, x, lags, h, s=s, y=y)
    r = oracle.corr(t, x, lags, "rectangle", h, s=s, y=y)
    assert r["count"].tolist() == cnt
    assert np.max(np.abs(r["c"] - np.array([float(v) for v in cs]))) < 1e-14
    # boundary hits were exercised: some pair separation equals tau +- h exactly
    sep = (s[None, :] - t[:, None]).ravel()
    assert np.any(np.isin(np.round((sep[None, :] - lags[:, None] + h) * 8), [0]))


@pytest.mark.parametrize("acf", [True, False])
def test_gaussian_direct_matches_50_digit_enumeration(acf):
    rng = _rng(7)
    t = np.sort(rng.uniform(0, 20, 9))
    x = rng.normal(size=9)
    lags = np.linspace(-3, 3, 13)
    kw = {}
    if not acf:
        kw = dict(s=np.sort(rng.uniform(0, 20, 8)), y=rng.normal(size=8))
    nums, dens, cs = oracle.exact_gaussian(t, x, lags, 0.7, **kw)
    r = oracle.corr(t, x, lags, "gaussian", 0.7, **kw)
    assert np.max(np.abs(r["b"] - np.array([float(v) for v in dens]))) < 1e-14
    assert np.max(np.abs(r["num"] - np.array([float(v) for v in nums]))) < 1e-14
    assert np.max(np.abs(r["c"] - np.array([float(v) for v in cs]))) < 1e-13


def test_regular_grid_reduces_to_textbook_estimator():
    """t_i = i, rectangle half-width 1/2, integer lags: the window holds exactly
    the pairs at separation k, so count_k = n - k and
    c_k = sum_t x_t x_{t+k} / (n - k) = n R(k) / (n - k), with R(k) the biased
    autocovariance of Eq. acf_regular of the standardised series."""
    rng = _rng(11)
    n = 200
    t = np.arange(n, dtype=np.float64)
    x = np.cumsum(rng.normal(size=n)) * 0.1 + rng.normal(size=n)
    lags = np.arange(0, 30, dtype=np.float64)
    r = oracle.corr(t, x, lags, "rectangle", 0.5)
    assert r["count"].tolist() == [n - k for k in range(30)]
    xs = (x - x.mean()) / x.std()
    full = np.correlate(xs, xs, mode="full")[n - 1:]       # sum_t x_t x_{t+k}
    R = full / n                                            # Eq. acf_regular
    ks = np.arange(30)
    np.testing.assert_allclose(r["c"], n * R[:30] / (n - ks), rtol=0, atol=1e-13)
    rl = oracle.corr(t, x, lags, "rectangle", 0.5, norm="lag0")
    np.testing.assert_allclose(rl["c"], (n * R[:30] / (n - ks)) / R[0], rtol=0, atol=1e-13)


def test_gaussian_pair_count_moments():
    """B(tau) = sum_pairs b(s_j - t_i - tau): integrating over tau gives
    n_x n_y (unit-mass kernel), the first moment sums the pair separations
    (the sign of the lag), the second adds h^2 per pair (the width)."""
    t = np.array([1.0, 2.5, 7.0])
    x = np.array([0.3, -1.0, 2.0])
    s = np.array([0.5, 4.0])
    y = np.array([1.0, -1.0])
    h = 0.8
    lags = np.linspace(-25, 25, 20001)
    dt = lags[1] - lags[0]
    r = oracle.corr(t, x, lags, "gaussian", h, s=s, y=y)
    B = r["b"]
    sep = (s[None, :] - t[:, None]).ravel()
    assert abs(B.sum() * dt - 6.0) < 1e-9
    assert abs((lags * B).sum() * dt - sep.sum()) < 1e-8
    assert abs((lags ** 2 * B).sum() * dt - (sep ** 2 + h * h).sum()) < 1e-7


@pytest.mark.parametrize("acf", [True, False])
def test_rectangle_windows_tiling_the_lag_axis_count_every_pair_once(acf):
    rng = _rng(13)
    t = np.sort(rng.uniform(0, 50, 60))
    x = rng.normal(size=60)
    h = 0.75
    kw = {} if acf else dict(s=np.sort(rng.uniform(0, 50, 45)), y=rng.normal(size=45))
    lags = 2 * h * np.arange(-40, 41)
    r = oracle.corr(t, x, lags, "rectangle", h, **kw)
    ny = 60 if acf else 45
    assert r["count"].sum() == 60 * ny


@pytest.mark.parametrize("kernel,h", [("gaussian", 0.6), ("rectangle", 0.6)])
def test_ccf_exchange_symmetry_and_acf_identity(kernel, h):
    rng = _rng(17)
    t = np.sort(rng.uniform(0, 40, 70))
    x = rng.normal(size=70)
    s = np.sort(rng.uniform(0, 40, 50))
    y = rng.normal(size=50)
    lags = np.linspace(-6, 6, 25)
    xy = oracle.corr(t, x, lags, kernel, h, s=s, y=y)
    yx = oracle.corr(s, y, -lags, kernel, h, s=t, y=x)
    np.testing.assert_allclose(xy["c"], yx["c"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(xy["b"], yx["b"], rtol=1e-14, atol=1e-14)
    assert np.array_equal(xy["count"], yx["count"])
    a = oracle.corr(t, x, lags, kernel, h)
    xx = oracle.corr(t, x, lags, kernel, h, s=t, y=x)
    np.testing.assert_allclose(a["c"], xx["c"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(a["c"], oracle.corr(t, x, -lags, kernel, h)["c"], rtol=0, atol=1e-13)
    al = oracle.corr(t, x, lags, kernel, h, norm="lag0")
    xxl = oracle.corr(t, x, lags, kernel, h, s=t, y=x, norm="lag0")
    np.testing.assert_allclose(al["c"], xxl["c"], rtol=0, atol=1e-13)


def test_affine_invariance():
    rng = _rng(19)
    t = np.sort(rng.uniform(0, 30, 50))
    x = rng.normal(size=50)
    s = np.sort(rng.uniform(0, 30, 40))
    y = rng.normal(size=40)
    lags = np.linspace(-5, 5, 11)
    base = oracle.corr(t, x, lags, "gaussian", 0.5, s=s, y=y)["c"]
    pos = oracle.corr(t, 3.0 * x + 7.0, lags, "gaussian", 0.5, s=s, y=y)["c"]
    neg = oracle.corr(t, -2.0 * x + 1.0, lags, "gaussian", 0.5, s=s, y=y)["c"]
    np.testing.assert_allclose(pos, base, rtol=0, atol=1e-13)
    np.testing.assert_allclose(neg, -base, rtol=0, atol=1e-13)


def test_shifted_copy_peaks_at_the_shift():
    """y = x read at times shifted by +tau0 (Sec. 3.1): the CCF peaks at +tau0
    with every point paired to its copy, count n and c = sum x_std^2 / n = 1."""
    rng = _rng(23)
    n = 80
    t = np.cumsum(rng.uniform(2.5, 4.0, n))   # min spacing 2.5 > 2h
    x = rng.normal(size=n)
    tau0 = 12.3
    s = t + tau0
    lags = np.round(np.arange(-30, 31) * 0.41, 10)
    k0 = int(np.argmin(np.abs(lags - tau0)))
    lags[k0] = tau0
    for kernel in ("rectangle", "gaussian"):
        r = oracle.corr(t, x, lags, kernel, 1.0, s=s, y=x)
        if kernel == "gaussian":
            assert int(np.argmax(r["c"])) == k0
        else:
            # lags within h of tau0 see the same pairs, so the maximum is a plateau
            assert r["c"][k0] == r["c"].max()
            assert r["count"][k0] == n
            assert abs(r["c"][k0] - 1.0) < 1e-14
    # a sign slip (eps = +1 for the CCF) would put the peak at -tau0
    r = oracle.corr(t, x, -lags, "rectangle", 1.0, s=s, y=x)
    assert r["count"][k0] != n


def test_windowed_scan_matches_direct_sum():
    rng = _rng(29)
    t = np.sort(rng.uniform(0, 100, 400))
    x = rng.normal(size=400)
    s = np.sort(rng.uniform(0, 100, 300))
    y = rng.normal(size=300)
    lags = np.linspace(-20, 20, 41)
    for kw in ({}, dict(s=s, y=y)):
        d = oracle.corr(t, x, lags, "rectangle", 0.9, **kw)
        w = oracle.corr(t, x, lags, "rectangle", 0.9, method="windowed", **kw)
        assert np.array_equal(d["count"], w["count"])
        np.testing.assert_allclose(w["c"], d["c"], rtol=0, atol=1e-13)
        d6 = oracle.corr(t, x, lags, "gaussian", 0.9, trunc_R=6, **kw)
        w6 = oracle.corr(t, x, lags, "gaussian", 0.9, method="windowed", trunc_R=6, **kw)
        assert np.array_equal(d6["count"], w6["count"])
        np.testing.assert_allclose(w6["c"], d6["c"], rtol=0, atol=1e-13)
        full = oracle.corr(t, x, lags, "gaussian", 0.9, **kw)
        w8 = oracle.corr(t, x, lags, "gaussian", 0.9, method="windowed", trunc_R=8, **kw)
        np.testing.assert_allclose(w8["c"], full["c"], rtol=0, atol=1e-12)
        # the paper's 6h window is visibly truncated at the 1e-10 level
        assert np.max(np.abs(d6["b"] - full["b"]) / full["b"]) > 1e-10


def test_time_shift_invariance_at_mjd_offsets():
    rng = _rng(31)
    t = np.sort(rng.uniform(0, 50, 120))
    x = rng.normal(size=120)
    lags = np.linspace(0, 10, 21)
    a = oracle.corr(t, x, lags, "gaussian", 0.4)["c"]
    b = oracle.corr(t + 60000.0, x, lags, "gaussian", 0.4)["c"]
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-10)


def test_degenerate_inputs_are_rejected():
    with pytest.raises(ValueError):
        oracle.standardise(np.ones(5))
    # lags with no pairs give c = 0 (clamped denominator) and b = 0
    t = np.array([0.0, 1.0, 2.0])
    r = oracle.corr(t, np.array([1.0, 2.0, 4.0]), np.array([50.0]), "rectangle", 0.5)
    assert r["count"][0] == 0 and r["c"][0] == 0.0 and r["b"][0] == 0.0
