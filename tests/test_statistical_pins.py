"""The oracle against the analytic correlation functions the paper validates with
(Sec. 3): a sinusoid, whose ACF is cos(2 pi tau / T); an Ornstein-Uhlenbeck
process sampled at irregular times, ACF exp(-|tau| / alpha); and a delayed noisy
copy of it, CCF kappa exp(-|tau - tau0| / alpha) (Eq. ou_theory_ccf).  The
kernel-weighted estimator averages the correlation over separations near tau, so
the expectations include that average in closed form (the kernel's Fourier
transform for the sinusoid; a negligible factor for the exponentials at h << alpha).
These are statistical checks on seeded realisations: tolerances are a few
standard errors of the estimate."""
import math

import numpy as np
import pytest

import oracle


def _ou(t, alpha, rng):
    """Exact OU sample path at sorted times t: unit variance, correlation time alpha."""
    x = np.empty(t.size)
    x[0] = rng.standard_normal()
    a = np.exp(-np.diff(t) / alpha)
    e = rng.standard_normal(t.size - 1) * np.sqrt(1.0 - a * a)
    for i in range(1, t.size):
        x[i] = a[i - 1] * x[i - 1] + e[i - 1]
    return x


@pytest.mark.parametrize("kernel", ["gaussian", "rectangle"])
def test_sinusoid_acf_is_the_damped_cosine(kernel):
    rng = np.random.default_rng(21)
    T, h = 20.0, 0.5
    t = np.sort(rng.uniform(0.0, 4000.0, 20000))
    x = np.cos(2 * np.pi * t / T + 0.7)
    lags = np.arange(0.0, 41.0, 1.0)
    got = oracle.corr(t, x, lags, kernel, h, method="windowed", trunc_R=8.0)["c"]
    f = 1.0 / T
    damp = math.exp(-2 * math.pi ** 2 * h * h * f * f) if kernel == "gaussian" else \
        math.sin(2 * math.pi * f * h) / (2 * math.pi * f * h)
    # deviations 0.005 (Gaussian) and 0.006 (rectangle); leaving out the Gaussian's
    # damping exp(-2 pi^2 h^2 / T^2) = 0.988 (sigma = h) would give 0.013
    np.testing.assert_allclose(got, damp * np.cos(2 * np.pi * lags / T), rtol=0, atol=0.008)


@pytest.mark.parametrize("kernel", ["gaussian", "rectangle"])
def test_ou_acf_is_the_exponential(kernel):
    rng = np.random.default_rng(22)
    alpha, h = 5.0, 0.5
    t = np.sort(rng.uniform(0.0, 20000.0, 100000))
    x = _ou(t, alpha, rng)
    lags = np.arange(1.0, 16.0)
    got = oracle.corr(t, x, lags, kernel, h, method="windowed", trunc_R=8.0)["c"]
    np.testing.assert_allclose(got, np.exp(-lags / alpha), rtol=0, atol=0.06)  # deviations about 0.025


def test_ou_ccf_of_a_delayed_noisy_copy():
    rng = np.random.default_rng(23)
    alpha, tau0, sig, h = 5.0, 7.0, 0.5, 0.5
    t = np.sort(rng.uniform(0.0, 20000.0, 100000))
    x = _ou(t, alpha, rng)
    s = t + tau0                                 # y(s) = x(s - tau0) + noise: y lags x by tau0
    y = x + sig * rng.standard_normal(t.size)
    lags = np.arange(-8.0, 23.0)
    got = oracle.corr(t, x, lags, "gaussian", h, s=s, y=y, method="windowed", trunc_R=8.0)["c"]
    kappa = 1.0 / math.sqrt(1.0 + sig * sig)
    np.testing.assert_allclose(got, kappa * np.exp(-np.abs(lags - tau0) / alpha), rtol=0, atol=0.06)
    assert lags[int(np.argmax(got))] == tau0
