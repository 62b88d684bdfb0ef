"""Thousands of lags in one batch: 3000 unsorted lags on [-200, 200] d (23 full
128-lag tiles of the tensor-core contraction plus a ragged one; 94 lag groups
of the scan, the last one partial), checked against the oracle on sampled lags:
the FP32 form within 1e-5, rectangle counts bit-exact and c within 1e-10."""
import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api, synth
from tests._gpu import to_np

pytestmark = pytest.mark.gpu


def test_three_thousand_lags_fp32_form_and_exact_scan():
    w = synth.light_curves(B=8, n_lo=300, n_hi=6000, K=8, seed=synth.BASE_SEED + 31)
    rng = np.random.default_rng(31)
    lags = rng.uniform(-200.0, 200.0, 3000)
    lags[17] = 0.0
    g = to_np(api.corr_batch(w.offs, w.t, w.x, lags, kernel="gaussian", h=0.5, path="spectral",
                             precision="fp32"))
    r = to_np(api.corr_batch(w.offs, w.t, w.x, lags, kernel="rectangle", h=0.5))
    assert g["c"].shape == (8, 3000) and r["count"].shape == (8, 3000)
    idx = np.concatenate([[0, 17, 2999], rng.choice(np.arange(1, 2999), 21, replace=False)])
    for b in range(w.B):
        sl = slice(int(w.offs[b]), int(w.offs[b + 1]))
        ref_g = oracle.corr(w.t[sl], w.x[sl], lags[idx], "gaussian", 0.5, method="windowed", trunc_R=8.0)
        ref_r = oracle.corr(w.t[sl], w.x[sl], lags[idx], "rectangle", 0.5, method="windowed")
        assert np.max(np.abs(g["c"][b, idx] - ref_g["c"])) <= 1e-5
        assert np.array_equal(r["count"][b, idx], ref_r["count"])
        assert np.max(np.abs(r["c"][b, idx] - ref_r["c"])) < 1e-10
