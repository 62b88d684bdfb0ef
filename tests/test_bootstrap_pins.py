"""Pins of the oracle's bootstrap resampler (CPU): the generator against its
published reference outputs, the structure of a replicate, and the law of the
multiplicities."""
import numpy as np

import oracle


def test_splitmix64_reference_outputs():
    # first three outputs of SplitMix64 started at 0 (the published reference values)
    assert [oracle.splitmix64(0, c) for c in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_replicate_is_a_sorted_multiset_of_the_points():
    for n in (2, 7, 1000):
        for r in (0, 1, 5):
            idx = oracle.bootstrap_indices(n, 12345, r)
            assert idx.size == n and idx.min() >= 0 and idx.max() < n
            assert np.all(np.diff(idx) >= 0)
    a, b = oracle.bootstrap_indices(500, 7, 0), oracle.bootstrap_indices(500, 7, 1)
    assert not np.array_equal(a, b)                      # replicates differ
    assert np.array_equal(a, oracle.bootstrap_indices(500, 7, 0))


def test_multiplicities_follow_binomial_n_1_over_n():
    """Each point's multiplicity is Binomial(n, 1/n): mean 1, variance 1 - 1/n;
    P(a point is left out) = (1 - 1/n)^n -> 1/e."""
    n, R = 400, 60
    m = np.stack([np.bincount(oracle.bootstrap_indices(n, 99, r), minlength=n) for r in range(R)])
    assert abs(m.mean() - 1.0) < 1e-12                   # exactly n draws per replicate
    assert abs(m.var() - (1 - 1 / n)) < 0.05
    assert abs((m == 0).mean() - (1 - 1 / n) ** n) < 0.01


def test_bootstrap_mean_tracks_the_full_sample_estimate():
    rng = np.random.default_rng(4)
    t = np.sort(rng.uniform(0, 300, 600))
    x = np.sin(2 * np.pi * t / 40) + 0.3 * rng.normal(size=t.size)
    lags = np.array([0.0, 10.0, 20.0])
    full = oracle.corr(t, x, lags, "rectangle", 2.0, method="windowed")["c"]
    reps = np.stack([oracle.bootstrap_corr(t, x, lags, r, 5, "rectangle", 2.0)["c"] for r in range(40)])
    assert np.all(np.abs(reps.mean(0) - full) < 4 * reps.std(0) / np.sqrt(40) + 0.02)
