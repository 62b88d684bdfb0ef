"""ncf_workspace_bytes: the device footprint of an evaluation before anything is
allocated.  Host arithmetic only, so these run without a GPU; the GPU test
(test_gpu_workspace.py) checks the bound against what plans really allocate."""
import pytest

from paper_2609_03866_b300 import api

LC = dict(n_x=113_916_677, B=4096, K=256, span=1460.0, max_abs_lag=200.0, h=0.5)


def ws(**k):
    return api.workspace_bytes(**k)


def test_light_curve_batch_footprints_are_positive_and_path_dependent():
    g32, pin = ws(**LC, kernel="gaussian", precision="fp32")
    rect, _ = ws(**LC, kernel="rectangle")
    assert g32 > 0 and pin > 0 and rect > 0
    # the exact scan keeps keys, quantised values and prefix sums: > 24 B per point
    assert rect > 24 * LC["n_x"]
    # the FP32 spectral path keeps B grids of >= 4 L / h complex FP32 cells
    assert g32 > LC["B"] * 4 * (LC["span"] / LC["h"]) * 8
    # a CCF spreads two series: more
    ccf, _ = ws(**dict(LC, n_y=LC["n_x"]), kernel="gaussian", precision="fp32")
    assert ccf > g32


def test_monotone_in_sizes_and_span():
    base = dict(LC, kernel="gaussian", precision="fp32")
    d0, _ = ws(**base)
    assert ws(**dict(base, K=1024))[0] > d0
    assert ws(**dict(base, n_x=2 * LC["n_x"]))[0] > d0
    assert ws(**dict(base, span=4 * LC["span"]))[0] > d0
    # the rectangle scan does not depend on the span
    r = dict(LC, kernel="rectangle")
    assert ws(**r)[0] == ws(**dict(r, span=10 * LC["span"]))[0]


def test_fp64_gaussian_auto_covers_both_paths():
    a = ws(**LC, kernel="gaussian", path="auto")[0]
    w = ws(**LC, kernel="gaussian", path="windowed")[0]
    s = ws(**LC, kernel="gaussian", path="spectral")[0]
    assert a == max(w, s)


def test_ccf_and_pearson_need_more():
    one = dict(n_x=100_000, B=1, K=200, span=3650.0, max_abs_lag=100.0, h=0.5, kernel="rectangle")
    acf = ws(**one)[0]
    ccf = ws(**dict(one, n_y=80_000))[0]
    lag0 = ws(**dict(one, n_y=80_000, norm="lag0"))[0]
    assert ccf > acf and lag0 > ccf


def test_refuses_what_the_calls_refuse():
    with pytest.raises(api.NcfError) as e:
        ws(n_x=3, B=2, K=4, span=1.0, max_abs_lag=1.0)      # a series of < 2 points
    assert e.value.status == 1
    with pytest.raises(api.NcfError) as e:
        ws(n_x=100, B=1, K=0, span=1.0, max_abs_lag=1.0)
    assert e.value.status == 1
    with pytest.raises(api.NcfError) as e:
        ws(n_x=100, B=1, K=4, span=float("nan"), max_abs_lag=1.0)
    assert e.value.status == 1
    with pytest.raises(api.NcfError) as e:                    # grid beyond 2^28 cells
        ws(n_x=100, B=1, K=4, span=1e9, max_abs_lag=1.0, kernel="gaussian", precision="fp32", h=0.01)
    assert e.value.status == 9
