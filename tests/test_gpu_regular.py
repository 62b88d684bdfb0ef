"""The classic-FFT path for regularly sampled data (ncf_corr_regular) against
the FP64 oracle evaluated on the times m * dt: rectangle counts bit-exact,
c within 1e-10 (Gaussian and rectangle), for gapless and gappy lattices,
repeated samples, CCFs and the Pearson normalisation."""
import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api
from tests._gpu import max_abs, to_np

pytestmark = pytest.mark.gpu


def lattice(n, keep=1.0, dup=0.0, seed=0, start=0):
    rng = np.random.default_rng(seed)
    m = np.arange(start, start + int(n / keep) + 1)
    m = m[rng.random(m.size) < keep][:n]
    if dup > 0:
        extra = rng.choice(m, int(dup * m.size))
        m = np.sort(np.concatenate([m, extra]))
    return m.astype(np.int64)


def ar1(n, seed):
    rng = np.random.default_rng(seed)
    e = rng.normal(size=n + 100)
    v = np.zeros_like(e)
    for i in range(1, e.size):
        v[i] = 0.8 * v[i - 1] + e[i]
    return v[100:]


@pytest.mark.parametrize("kernel,h", [("rectangle", 0.5), ("rectangle", 2.3), ("gaussian", 0.7), ("gaussian", 3.0)])
@pytest.mark.parametrize("keep,dup", [(1.0, 0.0), (0.7, 0.05)])
def test_acf_equals_the_oracle(kernel, h, keep, dup):
    m = lattice(3000, keep, dup, seed=1)
    x = ar1(m.size, 2)
    dt = 0.25
    lags = np.linspace(0.0, 60.0, 41) + 0.013
    got = to_np(api.corr_regular(m, x, dt, lags, kernel=kernel, h=h))
    ref = oracle.corr(m * dt, x, lags, kernel, h, method="windowed" if kernel == "rectangle" else "direct")
    if kernel == "rectangle":
        assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10
    assert max_abs(got["b"], ref["b"]) < 1e-9 * max(1.0, np.abs(ref["b"]).max())


@pytest.mark.parametrize("kernel", ["rectangle", "gaussian"])
def test_ccf_on_a_shared_lattice(kernel):
    m = lattice(2500, 0.8, seed=3)
    my = lattice(2000, 0.75, seed=4, start=40)
    x = ar1(m.size, 5)
    y = np.interp(my, m, x) + 0.3 * np.random.default_rng(6).normal(size=my.size)
    dt = 1.0 / 3.0
    lags = np.linspace(-40.0, 40.0, 33) + 0.07
    got = to_np(api.corr_regular(m, x, dt, lags, kernel=kernel, h=0.8, m_y=my, y=y))
    ref = oracle.corr(m * dt, x, lags, kernel, 0.8, s=my * dt, y=y,
                      method="windowed" if kernel == "rectangle" else "direct")
    if kernel == "rectangle":
        assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10


@pytest.mark.parametrize("ccf", [False, True])
def test_pearson_normalisation(ccf):
    m = lattice(1500, 0.9, seed=7)
    x = ar1(m.size, 8)
    lags = np.linspace(-10.0, 10.0, 21) + 0.01
    if ccf:
        my = lattice(1200, 0.85, seed=9)
        y = ar1(my.size, 10)
        got = to_np(api.corr_regular(m, x, 1.0, lags, kernel="gaussian", h=1.5, m_y=my, y=y, norm="lag0"))
        ref = oracle.corr(m * 1.0, x, lags, "gaussian", 1.5, s=my * 1.0, y=y, norm="lag0")
    else:
        got = to_np(api.corr_regular(m, x, 1.0, lags, kernel="rectangle", h=1.0, norm="lag0"))
        ref = oracle.corr(m * 1.0, x, lags, "rectangle", 1.0, norm="lag0", method="windowed")
    assert max_abs(got["c"], ref["c"]) < 1e-10


def test_boundary_ties_on_integer_times():
    """Integer steps, integer lags, integer half-width: every bound falls on a
    lattice point; both paths are exact there and must agree."""
    m = lattice(2000, 0.8, seed=11)
    x = ar1(m.size, 12)
    lags = np.arange(-15, 16, dtype=np.float64)
    for h in (1.0, 2.0):
        got = to_np(api.corr_regular(m, x, 1.0, lags, kernel="rectangle", h=h))
        ref = oracle.corr(m * 1.0, x, lags, "rectangle", h, method="windowed")
        assert np.array_equal(got["count"], ref["count"])
        assert max_abs(got["c"], ref["c"]) < 1e-10


def test_textbook_regular_acf_and_errors():
    """Gapless grid, h = dt/2, lags k dt: c_k = sum_t x_t x_(t+k) / (n - k) on
    standardised values (Eq. acf_regular without the 1/n factor)."""
    n = 4096
    x = ar1(n, 13)
    xs = (x - x.mean()) / x.std()
    lags = np.arange(0, 50, dtype=np.float64)
    got = to_np(api.corr_regular(np.arange(n), x, 1.0, lags, kernel="rectangle", h=0.5))
    want = np.array([np.dot(xs[: n - k], xs[k:]) / (n - k) for k in range(50)])
    assert np.array_equal(got["count"], n - np.arange(50))
    assert max_abs(got["c"], want) < 1e-11
    with pytest.raises(api.NcfError) as e:
        api.corr_regular(np.array([0, 2, 1, 3]), np.arange(4.0), 1.0, lags)
    assert e.value.name == "NCF_ENOTSORTED"
    with pytest.raises(api.NcfError) as e:
        api.corr_regular(np.arange(10), np.ones(10), 1.0, lags)
    assert e.value.name == "NCF_EDEGENERATE"
    with pytest.raises(api.NcfError) as e:
        api.corr_regular(np.arange(10), np.arange(10.0), 0.0, lags)
    assert e.value.name == "NCF_EINVAL"
