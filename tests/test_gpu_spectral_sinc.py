"""The spectral-sinc rectangle (the rectangle on the spectral path): the
cross-spectrum times sin(2 pi f h)/(pi f) summed over |m| <= L/(h tol) modes.
Its error against the exact estimator is reported, not gated at the FP64
tolerance: the truncated transform of a box misweights pairs within about
L/M of a window edge, so the pair count B and the numerator carry errors of
order tol (relative), and c of order tol.  The tests check that order and
that the error falls as tol does."""
import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api
from tests._gpu import to_np

pytestmark = pytest.mark.gpu


def _series(n, span, seed, phase=0.0):
    rng = np.random.default_rng(seed)
    t = np.sort(rng.uniform(0.0, span, n)) + phase
    x = np.sin(t / 4.0) + 0.5 * rng.standard_normal(n)
    return t, x


def _errors(got, ref):
    dc = np.abs(got["c"] - ref["c"]).max()
    db = (np.abs(got["b"] - ref["b"]) / np.maximum(ref["b"], 1.0)).max()
    return dc, db


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_acf_error_is_of_order_tol_and_falls_with_it(precision):
    t, x = _series(3000, 300.0, 1)
    lags = np.linspace(0.0, 40.0, 41)
    ref = oracle.corr(t, x, lags, "rectangle", 0.5, method="windowed")
    errs = []
    for tol in (1e-3, 1e-4):
        got = to_np(api.corr(t, x, lags, kernel="rectangle", h=0.5, path="spectral", precision=precision, tol=tol))
        dc, db = _errors(got, ref)
        print("acf", precision, tol, dc, db)
        assert dc < 20 * tol and db < 20 * tol
        assert np.all(got["count"] == 0)
        errs.append(max(dc, db))
    assert errs[1] < errs[0] / 3


def test_ccf_and_pearson_error_is_of_order_tol():
    t, x = _series(2500, 250.0, 2)
    s, y = _series(2000, 220.0, 3, phase=11.0)
    lags = np.linspace(-30.0, 30.0, 37)
    for norm in ("none", "lag0"):
        ref = oracle.corr(t, x, lags, "rectangle", 0.75, s=s, y=y, norm=norm, method="windowed")
        got = to_np(api.corr(t, x, lags, kernel="rectangle", h=0.75, s=s, y=y, norm=norm, path="spectral",
                             tol=1e-4))
        dc, db = _errors(got, ref)
        print("ccf", norm, dc, db)
        assert dc < 2e-3 and db < 2e-3
