"""Pins of the oracle of the paper's NUFFT variant (Algorithms 1-4 with the
smoothing step S_h) against routines and identities outside the oracle."""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from oracle import paper_nufft as pn


# --- S_h against scipy.ndimage (the reading of the filter) -------------------

@pytest.mark.parametrize("n", [1, 2, 3, 7, 40])
def test_gaussian_filter_is_scipy_default(n):
    a = np.random.default_rng(n).standard_normal(n)
    for h in (0.3, 0.5, 1.0, 1.3, 2.5, 7.0):
        ref = ndi.gaussian_filter1d(a, sigma=h, mode="reflect", truncate=4.0)
        np.testing.assert_allclose(pn.smooth(a, "gaussian", h), ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 40])
def test_box_filter_is_scipy_uniform_filter(n):
    a = np.random.default_rng(100 + n).standard_normal(n)
    for h in (0.5, 1.0, 1.25, 1.5, 2.0, 3.3, 9.0):
        ref = ndi.uniform_filter1d(a, size=pn.box_size(h), mode="reflect")
        np.testing.assert_allclose(pn.smooth(a, "rectangle", h), ref, rtol=0, atol=1e-13)


def test_box_size_rounds_half_to_even():
    # round(2h) as the paper's Python package rounds: 2.5 -> 2, 3.5 -> 4
    assert [pn.box_size(h) for h in (0.5, 1.0, 1.25, 1.5, 1.75)] == [1, 2, 2, 3, 4]
    with pytest.raises(ValueError):
        pn.smooth(np.ones(5), "rectangle", 0.2)


# --- the transforms against numpy's FFT on uniform points ---------------------

@pytest.mark.parametrize("N", [16, 17])
def test_type1_on_uniform_points_is_an_inverse_dft(N):
    c = np.random.default_rng(N).standard_normal(N)
    tt = 2.0 * np.pi * np.arange(N) / N
    F = pn.nufft1d1(tt, c, N)
    k = pn.modes(N)
    ref = N * np.fft.ifft(c)[k % N]          # sum_j c_j exp(+2 pi i k j / N)
    np.testing.assert_allclose(F, ref, rtol=0, atol=1e-11)
    assert k[0] == -(N // 2) and k[-1] == (N + 1) // 2 - 1 and k.size == N


@pytest.mark.parametrize("N", [16, 17])
def test_type2_on_uniform_points_is_a_forward_dft(N):
    rng = np.random.default_rng(7 + N)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    taut = 2.0 * np.pi * np.arange(N) / N
    g = np.zeros(N, dtype=complex)
    g[pn.modes(N) % N] = f
    np.testing.assert_allclose(pn.nufft1d2(taut, f, N), np.fft.fft(g), rtol=0, atol=1e-11)


# --- c_raw through the spectra equals a pair sum of Dirichlet kernels ---------

def _dirichlet(theta, N):
    """sum_{k=-floor(N/2)}^{ceil(N/2)-1} exp(i k theta) in closed form."""
    a = N // 2
    z = np.exp(1j * theta)
    out = np.empty(theta.shape, dtype=complex)
    small = np.abs(np.sin(theta / 2.0)) < 1e-12
    out[~small] = np.exp(-1j * a * theta[~small]) * (np.exp(1j * N * theta[~small]) - 1.0) / (z[~small] - 1.0)
    out[small] = N
    return out


@pytest.mark.parametrize("N1", [64, 65])
def test_raw_correlation_is_a_dirichlet_pair_sum(N1):
    rng = np.random.default_rng(N1)
    t = np.sort(rng.uniform(3.0, 40.0, 23))
    s = np.sort(rng.uniform(0.0, 35.0, 19))
    x, y = rng.standard_normal(23), rng.standard_normal(19)
    taus = np.array([-7.3, -1.0, 0.0, 0.4, 2.5, 11.0])
    t_min = min(t.min(), s.min())
    span = max(t.max(), s.max()) - t_min
    L, N, t_c = pn.padded_domain(t_min, span, taus, 23, N1)
    F1 = pn.nufft1d1(np.pi + 2 * np.pi * (t - t_c) / L, x, N)
    F2 = pn.nufft1d1(np.pi + 2 * np.pi * (s - t_c) / L, y, N)
    got = pn.raw_correlation(F1, F2, taus, L, N)
    d = s[None, None, :] - t[None, :, None] - taus[:, None, None]   # s_j - t_i - tau
    ref = np.einsum("i,j,kij->k", x, y, np.real(_dirichlet(2 * np.pi * d / L, N)))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


# --- Algorithm 1 -------------------------------------------------------------

def test_padded_domain_worked_example():
    L, N1, t_c = pn.padded_domain(10.0, 100.0, np.array([-30.0, 0.0, 5.0]), 50)
    assert (L, N1, t_c) == (160.0, 2560, 60.0)
    # 32 * 1 * 65 / 64 = 32.5 exactly: rounds half to even
    assert pn.padded_domain(0.0, 64.0, np.array([0.0, 0.5]), 1)[1] == 32
    assert pn.padded_domain(0.0, 64.0, np.array([0.0, 0.5]), 1, N1=77)[1] == 77


# --- whole estimators ----------------------------------------------------------

def _daily(n, seed, gap_every=0):
    rng = np.random.default_rng(seed)
    t = np.arange(n, dtype=np.float64)
    if gap_every:
        t = t[(np.arange(n) % gap_every) != gap_every - 1]
    v = np.zeros(t.size)
    for i in range(1, t.size):
        v[i] = 0.8 * v[i - 1] + rng.standard_normal()
    return t, v


@pytest.mark.parametrize("kernel,h", [("gaussian", 1.0), ("rectangle", 1.5)])
def test_delayed_copy_peaks_at_plus_delay(kernel, h):
    # y is x delayed by 7 days: the CCF peak sits at lag +7 (y lags x)
    t, v = _daily(260, 3)
    tt = t[:-7]
    x, y = v[7:], v[:-7]          # on common times: y(t) = x(t - 7)
    lags = np.arange(-15.0, 16.0)
    r = pn.ccf(tt, x, tt, y, lags, kernel, h)
    assert lags[int(np.argmax(r["c"]))] == 7.0


@pytest.mark.parametrize("kernel,h", [("gaussian", 0.7), ("rectangle", 1.2), ("rectangle", 1.5)])
def test_acf_equals_ccf_of_itself_on_the_symmetric_array(kernel, h):
    # lags +-1 .. +-n_h plus the prepended 0 form Algorithm 3's symmetric array,
    # so Algorithm 4's lag-0 entry is Algorithm 3's interior scale and the two
    # estimators coincide (the pair counts are even in tau as long as no pair
    # sits on a window edge: h is not an integer, so the self-pairs never do)
    rng = np.random.default_rng(5)
    t = np.sort(rng.uniform(0.0, 120.0, 150))
    x = np.sin(t / 3.0) + 0.3 * rng.standard_normal(150)
    n_h = max(math.ceil(4 * h) + 2, 5)
    lags = np.concatenate([np.arange(-n_h, 0.0), np.arange(1.0, n_h + 1)])
    a = pn.acf(t, x, lags, kernel, h)
    c = pn.ccf(t, x, t, x, lags, kernel, h)
    np.testing.assert_allclose(a["c"], c["c"], rtol=0, atol=1e-12)
    if kernel == "gaussian" or pn.box_size(h) % 2 == 1:
        # a symmetric filter keeps the ACF even in tau; an even box size (offsets
        # -size/2 .. size/2 - 1) does not
        np.testing.assert_allclose(a["c"], a["c"][::-1], rtol=0, atol=1e-12)


# On integer times with unit lag spacing and an integer period L, a grid size N1
# that is a multiple of L makes the Dirichlet kernel vanish at every nonzero
# integer separation (exp(i N1 theta) = 1 at theta = 2 pi m / L).  The raw
# correlation is then N1 times the exact lagged-product sums, the array
# smoothing is the kernel (a box of 3 entries is the count window [-1.5, 1.5];
# the Gaussian is sampled at the integers and renormalised over |j| <= 4h), and
# the variant is the kernel estimator itself -- exactly for the box, to the
# Gaussian's tail beyond 4h (about 4e-6 relative) otherwise -- at every lag far
# enough from the array ends to escape the reflecting filter's edge artifact.
_TOL = {"gaussian": 1e-5, "rectangle": 1e-12}


def _inner(lags, kernel, h):
    r = int(4 * h + 0.5) if kernel == "gaussian" else pn.box_size(h) // 2
    return np.abs(lags) <= np.abs(lags).max() - r - 1


def _multiple_of_L(fn, *args):
    L, N1 = (lambda r: (r["L"], r["N1"]))(fn(*args))
    assert L == int(L)
    return fn(*args, N1=int(np.ceil(N1 / L)) * int(L))


@pytest.mark.parametrize("kernel,h", [("gaussian", 1.0), ("rectangle", 1.5)])
def test_integer_day_acf_is_the_kernel_estimator(kernel, h):
    t, x = _daily(400, 11, gap_every=9)
    lags = np.concatenate([np.arange(-24.0, 0.0), np.arange(1.0, 25.0)])
    ex = oracle.corr(t, x, lags, kernel, h, norm="lag0", method="windowed", trunc_R=6.0)
    var = _multiple_of_L(pn.acf, t, x, lags, kernel, h)
    inner = _inner(lags, kernel, h)
    np.testing.assert_allclose(var["c"][inner], ex["c"][inner], rtol=0, atol=_TOL[kernel])
    np.testing.assert_allclose(var["b"], ex["b"], rtol=1e-12)
    # with the default N1 the leakage is still small but visible
    dflt = pn.acf(t, x, lags, kernel, h)
    assert np.abs(dflt["c"] - ex["c"])[inner].max() < 1e-2


@pytest.mark.parametrize("kernel,h", [("gaussian", 1.0), ("rectangle", 1.5)])
def test_integer_day_ccf_is_the_kernel_estimator(kernel, h):
    # two gappy daily series, y a delayed noisy copy of x: the interior scales
    # of Algorithm 3 stand for sqrt(ACF_x(0) ACF_y(0))
    t, v = _daily(420, 12)
    rng = np.random.default_rng(13)
    keep_x = (np.arange(t.size - 5) % 7) != 3
    keep_y = (np.arange(t.size - 5) % 11) != 5
    tx, x = t[:-5][keep_x], v[5:][keep_x]
    ty, y = t[:-5][keep_y], v[:-5][keep_y] + 0.3 * rng.standard_normal(keep_y.sum())
    lags = np.concatenate([np.arange(-20.0, 0.0), np.arange(1.0, 21.0)])
    ex = oracle.corr(tx, x, lags, kernel, h, s=ty, y=y, norm="lag0", method="windowed", trunc_R=6.0)
    var = _multiple_of_L(pn.ccf, tx, x, ty, y, lags, kernel, h)
    inner = _inner(lags, kernel, h)
    np.testing.assert_allclose(var["c"][inner], ex["c"][inner], rtol=0, atol=_TOL[kernel])
    np.testing.assert_allclose(var["b"], ex["b"], rtol=1e-12)
    assert lags[int(np.argmax(var["c"]))] == 5.0
