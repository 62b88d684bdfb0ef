"""Pins of the oracle's Hanning kernel (the Hann window of half-width h and unit
mass, the reading of the kernel Sec. 2.3 names): exact enumeration, the
classical estimator it reduces to on a regular grid, its mass and compact
support, and O1 = O2."""
import numpy as np

import oracle


def test_exact_enumeration_dozen_points():
    rng = np.random.default_rng(1)
    t = np.sort(rng.uniform(0, 10, 12))
    x = rng.normal(size=12)
    lags = np.array([0.0, 0.7, 1.9, -2.3])
    _, _, cs = oracle.exact_hanning(t, x, lags, 1.3)
    got = oracle.corr(t, x, lags, "hanning", 1.3)["c"]
    assert np.max(np.abs(got - np.array([float(c) for c in cs]))) < 1e-14
    s = np.sort(rng.uniform(0, 10, 9))
    y = rng.normal(size=9)
    _, _, cs = oracle.exact_hanning(t, x, lags, 0.9, s=s, y=y)
    got = oracle.corr(t, x, lags, "hanning", 0.9, s=s, y=y)["c"]
    assert np.max(np.abs(got - np.array([float(c) for c in cs]))) < 1e-14


def test_regular_grid_with_h_equal_to_the_step_is_the_classical_estimator():
    """t_i = i, h = 1: at integer lags only d = 0 has weight (cos^2(pi/2) = 0 at
    d = +-1), so c_k = sum_t x_t x_(t+k) / (n - k) on standardised values."""
    rng = np.random.default_rng(2)
    n = 500
    x = np.cumsum(rng.normal(size=n)) * 0.1 + rng.normal(size=n)
    xs = (x - x.mean()) / x.std()
    lags = np.arange(0, 30, dtype=np.float64)
    r = oracle.corr(np.arange(n, dtype=np.float64), x, lags, "hanning", 1.0)
    want = np.array([np.dot(xs[: n - k], xs[k:]) / (n - k) for k in range(30)])
    assert np.max(np.abs(r["c"] - want)) < 1e-12
    # b = sum of weights = (n - k) * 1/h, plus the two zero-weight neighbours counted
    assert np.allclose(r["b"], (n - lags))


def test_unit_mass_and_compact_support():
    """On a fine regular grid (step 1e-3), the weights in one point's window at lag 0
    sum to 1/step (unit mass) except within h of the ends.  Points added 100 d away,
    1 d apart, add only their own self pairs: 1/h each to b."""
    step, h = 1e-3, 0.5
    t = np.arange(0, 20, step)
    x = np.sin(t) + 0.1 * np.cos(7 * t)
    r = oracle.corr(t, x, np.array([0.0]), "hanning", h, method="windowed")
    # edge points at distance u < h from an end keep int_{-u}^{h} of the unit mass
    u = np.linspace(0, h, 2001)
    edge = np.mean(0.5 + u / (2 * h) + np.sin(np.pi * u / h) / (2 * np.pi))
    want = (t.size - 2 * h / step) + (2 * h / step) * edge
    assert abs(r["b"][0] * step - want * 1.0) / want < 2e-3
    far = t[-1] + 100.0 + np.arange(10.0)
    r2 = oracle.corr(np.concatenate([t, far]), np.concatenate([x, np.ones(10)]), np.array([0.0]), "hanning", h,
                     method="windowed")
    assert abs(r2["b"][0] - (r["b"][0] + 10 / h)) < 1e-6 * r["b"][0]


def test_windowed_equals_direct():
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 300, 800))
    x = rng.normal(size=800)
    lags = np.linspace(-20, 20, 17)
    a = oracle.corr(t, x, lags, "hanning", 1.7, method="direct")
    b = oracle.corr(t, x, lags, "hanning", 1.7, method="windowed")
    assert np.array_equal(a["count"], b["count"])
    assert np.max(np.abs(a["c"] - b["c"])) < 1e-12
