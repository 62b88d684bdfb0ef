"""Bootstrap replicates drawn on the GPU (ncf_corr_bootstrap) equal the
oracle's replicates (its own SplitMix64 resampler) evaluated by the oracle:
rectangle counts bit-exact, FP64 c within 1e-10, the FP32 form within 1e-5."""
import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import api, synth
from tests._gpu import max_abs, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def series():
    return synth.light_curves(B=1, n_lo=3000, n_hi=3001, K=24, seed=synth.BASE_SEED + 41)


@pytest.mark.parametrize("kernel,precision,tol", [("rectangle", "fp64", 1e-10), ("gaussian", "fp64", 1e-10),
                                                  ("gaussian", "fp32", 1e-5)])
def test_acf_replicates_equal_the_oracle(series, kernel, precision, tol):
    w = series
    seed = 0x1234_5678_9ABC_DEF0
    got = to_np(api.corr_bootstrap(w.t, w.x, w.lags, n_boot=6, seed=seed, kernel=kernel, h=0.5,
                                   precision=precision, path="spectral" if kernel == "gaussian" else "auto"))
    for r in range(6):
        ref = oracle.bootstrap_corr(w.t, w.x, w.lags, r, seed, kernel, 0.5,
                                    method="windowed" if kernel == "rectangle" else "direct")
        if kernel == "rectangle":
            assert np.array_equal(got["count"][r], ref["count"])
        assert max_abs(got["c"][r], ref["c"]) < tol, r


def test_ccf_replicates_draw_each_side_independently():
    c = synth.ou_ccf(nA=4000, nB=3200, K=21)
    seed = 77
    got = to_np(api.corr_bootstrap(c.t, c.x, c.lags, n_boot=4, seed=seed, kernel="rectangle", h=0.5,
                                   s=c.s, y=c.y))
    for r in range(4):
        ref = oracle.bootstrap_corr(c.t, c.x, c.lags, r, seed, "rectangle", 0.5, s=c.s, y=c.y)
        assert np.array_equal(got["count"][r], ref["count"])
        assert max_abs(got["c"][r], ref["c"]) < 1e-10


def test_many_replicates_and_argument_errors(series):
    w = series
    got = to_np(api.corr_bootstrap(w.t, w.x, w.lags, n_boot=512, seed=3, kernel="gaussian", h=0.5,
                                   precision="fp32", path="spectral"))
    full = to_np(api.corr(w.t, w.x, w.lags, kernel="gaussian", h=0.5, precision="fp32", path="spectral"))
    assert got["c"].shape == (512, w.lags.size) and np.all(np.isfinite(got["c"]))
    # the bootstrap distribution is centred near the full-sample estimate
    assert np.all(np.abs(np.median(got["c"], axis=0) - full["c"]) < 4 * got["c"].std(axis=0) + 1e-3)
    for bad in (dict(n_boot=0), dict(n_boot=-1)):
        with pytest.raises(api.NcfError) as e:
            api.corr_bootstrap(w.t, w.x, w.lags, seed=1, **bad)
        assert e.value.name == "NCF_EINVAL"
    with pytest.raises(api.NcfError) as e:
        api.corr_bootstrap(w.t[:1], w.x[:1], w.lags, n_boot=2)
    assert e.value.name == "NCF_EINVAL"
