"""The oracle against a worked example enumerated by hand (tests/golden/):
integer times with a gap, small integer values and the rectangle kernel, where
every estimate is an exact rational (times 1/sqrt(5) for the CCF) and every
pair count an exact integer.  The fixture pins the lag sign convention (tau > 0:
y lags x), the closed window edges, the self-pairs of the ACF, ddof 0 and the
lag-0 normalisation of Algorithm 4, independently of the oracle's code."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rectangle_hand_example.json")


def load_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def expected(case):
    """(c, count) of a case: c from its exact rationals, divided by sqrt(c_times_sqrt)."""
    root = math.sqrt(case["c_times_sqrt"])
    c = np.array([float(Fraction(v)) / root for v in case["c"]])
    return c, np.array(case["count"], dtype=np.int64)


def args(case):
    a = dict(kernel="rectangle", h=case["h"], norm=case["norm"])
    if "s" in case:
        a.update(s=np.array(case["s"], dtype=np.float64), y=np.array(case["y"], dtype=np.float64))
    return (np.array(case["t"], dtype=np.float64), np.array(case["x"], dtype=np.float64),
            np.array(case["lags"], dtype=np.float64)), a


def test_fixture_is_consistent():
    for case in load_cases():
        n = len(case["lags"])
        assert len(case["count"]) == n and len(case["c"]) == n, case["name"]
        assert len(case["t"]) == len(case["x"])
        # a lag without pairs has the estimate 0 (the clamp of the denominator)
        for cnt, v in zip(case["count"], case["c"]):
            assert cnt > 0 or Fraction(v) == 0


@pytest.mark.parametrize("method", ["direct", "windowed"])
@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_oracle_reproduces_the_hand_enumeration(case, method):
    pos, kw = args(case)
    got = oracle.corr(*pos, method=method, **kw)
    c, count = expected(case)
    assert np.array_equal(got["count"], count)
    assert np.array_equal(got["b"], count.astype(np.float64))   # the rectangle weighs each pair 1
    np.testing.assert_allclose(got["c"], c, rtol=0, atol=1e-15)
