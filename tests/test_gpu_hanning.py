"""The Hanning kernel (Hann window of half-width h, unit mass) on the FP64
windowed path and on the regular-grid path, against the FP64 oracle: c within
1e-10, pair counts (pairs in the closed window) bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api, synth
from tests._gpu import max_abs, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("h", [1.0, 0.37])
def test_acf_ar1(h):
    w = synth.ar1_acf()
    ref = oracle.corr(w.t, w.x, w.lags, "hanning", h)
    got = to_np(api.corr(w.t, w.x, w.lags, kernel="hanning", h=h))
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10
    assert max_abs(got["b"], ref["b"]) < 1e-9 * max(1.0, np.abs(ref["b"]).max())


def test_ccf_batch_pearson_and_ties():
    c = synth.ou_ccf(nA=6000, nB=4800, K=41)
    ref = oracle.corr(c.t, c.x, c.lags, "hanning", 0.5, s=c.s, y=c.y, method="windowed")
    got = to_np(api.corr(c.t, c.x, c.lags, kernel="hanning", h=0.5, s=c.s, y=c.y))
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10
    w = synth.light_curves(B=7, n_lo=300, n_hi=5000, K=30)
    got = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="hanning", h=0.5, norm="lag0"))
    for b in range(w.B):
        sl = slice(int(w.offs[b]), int(w.offs[b + 1]))
        ref = oracle.corr(w.t[sl], w.x[sl], w.lags, "hanning", 0.5, norm="lag0", method="windowed")
        assert max_abs(got["c"][b], ref["c"]) < 1e-10
    # integer times and lags, h integer: bounds on sample times; weights vanish there
    rng = np.random.default_rng(4)
    t = np.sort(rng.choice(3000, 1200, replace=False)).astype(np.float64)
    x = rng.normal(size=t.size)
    lags = np.arange(-10, 11, dtype=np.float64)
    ref = oracle.corr(t, x, lags, "hanning", 2.0)
    got = to_np(api.corr(t, x, lags, kernel="hanning", h=2.0))
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10


def test_regular_grid_and_unsupported_forms():
    rng = np.random.default_rng(5)
    m = np.sort(rng.choice(20000, 9000, replace=False)).astype(np.int64)
    x = rng.normal(size=m.size)
    lags = np.linspace(0, 40, 23) + 0.03
    got = to_np(api.corr_regular(m, x, 0.5, lags, kernel="hanning", h=1.3))
    ref = oracle.corr(m * 0.5, x, lags, "hanning", 1.3, method="windowed")
    assert np.array_equal(got["count"], ref["count"])
    assert max_abs(got["c"], ref["c"]) < 1e-10
    w = synth.ar1_acf(n=500, K=5)
    for kw in (dict(path="spectral"), dict(precision="fp32")):
        with pytest.raises(api.NcfError) as e:
            api.corr(w.t, w.x, w.lags, kernel="hanning", h=1.0, **kw)
        assert e.value.name == "NCF_EUNSUPPORTED"
