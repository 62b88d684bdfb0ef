"""Parity at the benchmark's full size and launch configuration: 4096 light
curves (n log-uniform in [200, 2e5], 113.9 M points) x 256 lags, the Gaussian
through the batched FP32 form and the rectangle through the exact scan, one
batched call each (as the benchmark times them).  Sampled outputs are checked
against the FP64 oracle one series at a time: rectangle counts bit-exact and c
within 1e-10, the Gaussian FP32 form within 1e-5 (window 8h in the oracle,
whose truncation is below 1e-14)."""
import os

import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api, synth
from tests._gpu import to_np

pytestmark = pytest.mark.gpu
H = 0.5


@pytest.fixture(scope="module")
def batch():
    return synth.light_curves(B=4096, K=256)


def test_light_curves_4096_x_256_sampled_against_the_oracle(batch):
    w = batch
    g = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=H, path="spectral",
                             precision="fp32"))
    r = to_np(api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="rectangle", h=H))
    assert g["c"].shape == (4096, 256) and np.all(np.isfinite(g["c"])) and np.all(np.isfinite(r["c"]))
    rng = np.random.default_rng(2026)
    sizes = np.diff(w.offs)
    # the largest series, the smallest, and a random sample
    pick = np.unique(np.concatenate([[int(np.argmax(sizes)), int(np.argmin(sizes))],
                                     rng.choice(w.B, 14, replace=False)]))
    for b in pick:
        sl = slice(int(w.offs[b]), int(w.offs[b + 1]))
        ks = np.sort(rng.choice(256, 6, replace=False))
        ref_r = oracle.corr(w.t[sl], w.x[sl], w.lags[ks], "rectangle", H, method="windowed")
        assert np.array_equal(r["count"][b, ks], ref_r["count"]), b
        assert np.max(np.abs(r["c"][b, ks] - ref_r["c"])) < 1e-10, b
        ref_g = oracle.corr(w.t[sl], w.x[sl], w.lags[ks], "gaussian", H, method="windowed", trunc_R=8.0)
        assert np.max(np.abs(g["c"][b, ks] - ref_g["c"])) < 1e-5, b


@pytest.fixture(scope="module")
def fp64_gauss(batch):
    w = batch
    return api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=H, path="spectral", precision="fp64")


@pytest.mark.parametrize("spread", [None, 0, 1, 2, 3])
def test_light_curves_4096_x_256_every_fp32_value_within_1e5_of_the_fp64_path(batch, fp64_gauss, spread):
    """Every one of the 4096 x 256 values of the batched FP32 form against the FP64
    spectral path on the same batch, which the oracle pins within 1e-10 (the
    sampled test above and the spectral parity tests): with the shapes the tuner
    picks, and with each spreading (CTAs of 4096 or 2048 points, tile sums in FP32
    or in fixed point) pinned beside the tensor-core contraction."""
    w = batch
    old = os.environ.get("NCF_SPEC_VARIANT")
    if spread is not None:
        os.environ["NCF_SPEC_VARIANT"] = str(4 * spread)
    try:
        f32 = api.corr_batch(w.offs, w.t, w.x, w.lags, kernel="gaussian", h=H, path="spectral",
                             precision="fp32")
    finally:
        if old is None:
            os.environ.pop("NCF_SPEC_VARIANT", None)
        else:
            os.environ["NCF_SPEC_VARIANT"] = old
    d = (f32["c"] - fp64_gauss["c"]).abs()
    assert d.numel() == 4096 * 256
    assert float(d.max()) < 1e-5, float(d.max())
    assert float((f32["b"] / fp64_gauss["b"] - 1).abs().max()) < 1e-5
