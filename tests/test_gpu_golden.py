"""The CUDA rectangle paths against the worked example enumerated by hand
(tests/golden/): exact pair counts, and estimates within the scan's fixed-point
quantisation of the standardised values (2^-27 relative at least, far below
1e-10 at these magnitudes)."""
import numpy as np
import pytest

from paper_2609_03866_b300 import api
from tests._gpu import to_np
from tests.test_golden import args, expected, load_cases

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.mark.parametrize("path", ["auto", "windowed"])
@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_single_call_reproduces_the_hand_enumeration(case, path):
    pos, kw = args(case)
    got = to_np(api.corr(*pos, path=path, **kw))
    c, count = expected(case)
    assert np.array_equal(got["count"], count)
    assert np.array_equal(got["b"], count.astype(np.float64))
    np.testing.assert_allclose(got["c"], c, rtol=0, atol=TOL)


@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_batch_of_three_copies_reproduces_the_hand_enumeration(case):
    # the batched scan: three copies of the series, CSR-packed, one lag grid
    (t, x, lags), kw = args(case)
    n = t.size
    offs = np.array([0, n, 2 * n, 3 * n], dtype=np.int64)
    if "s" in kw:
        s, y = kw.pop("s"), kw.pop("y")
        m = s.size
        kw.update(offs_y=np.array([0, m, 2 * m, 3 * m], dtype=np.int64), s=np.tile(s, 3), y=np.tile(y, 3))
    got = to_np(api.corr_batch(offs, np.tile(t, 3), np.tile(x, 3), lags, **kw))
    c, count = expected(case)
    for b in range(3):
        assert np.array_equal(got["count"][b], count)
        np.testing.assert_allclose(got["c"][b], c, rtol=0, atol=TOL)
