"""One process per GPU: which series a rank evaluates, and the rank bookkeeping
around a timed region.

Series are independent units of the estimator (Sec. 2.3: every c_k of one
series or pair depends on that series or pair only), so a batch splits across
ranks with no exchange on the data path.  Two ways are offered:

* weak scaling -- every rank evaluates its own batch (``rank_seed``);
* strong scaling -- one batch is cut into contiguous series ranges of about
  equal cost (``partition_series``), each rank evaluates its range
  (``sub_batch``) and rank 0 gathers the rows (``gather_rows``).

The only collectives are host-side bookkeeping: barriers, the maximum of the
per-rank times and the gather of result rows (``torch.distributed``; NCCL on
GPUs, gloo in the CPU tests).

One very long series splits too (``split_series``): the estimator's sums are
additive over the outer points (Eq. kernel_estimator, N_k = sum_j y_j sum_i
x_i b(s_j - t_i - tau_k), and likewise B_k and the pair counts), so each rank
takes a contiguous range of outer points and the inner points within reach of
it (max|tau| plus the kernel's half-width: a halo), evaluates its partial sums
and the ranks add them: exact integer pair counts, FP64 sums.  The
standardisation of the whole series is pooled from the ranges' own statistics
(Chan, Golub and LeVeque's pairwise update) before any rank evaluates.  The
exchanges are an all-gather of three numbers per rank and series and an
all-reduce of 3K numbers; no point crosses ranks.
"""
from __future__ import annotations

import os

import numpy as np


def dist_env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s own batch under weak scaling."""
    return int(base_seed) + int(rank)


def series_cost(offs, K: int, offs_y=None) -> np.ndarray:
    """Work of each series: (outer points) x K items plus a fixed per-series term
    (launch tiles, statistics)."""
    offs = np.asarray(offs, dtype=np.int64)
    n = np.diff(offs if offs_y is None else np.asarray(offs_y, dtype=np.int64)).astype(np.float64)
    return n * float(max(K, 1)) + 2048.0 * float(max(K, 1))


def partition_series(offs, K: int, world: int, offs_y=None):
    """Contiguous series ranges [(b0, b1)] per rank, cut where the cumulative cost
    crosses r / world of the total.  Every series lands on exactly one rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = series_cost(offs, K, offs_y)
    B = cost.size
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(cum, total * r / world, side="left")))
    cuts.append(B)
    cuts = np.maximum.accumulate(np.minimum(np.asarray(cuts), B))
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(world)]


def sub_batch(offs, b0: int, b1: int):
    """CSR offsets of series [b0, b1) rebased to 0, and the point slice they cover."""
    offs = np.asarray(offs, dtype=np.int64)
    lo, hi = int(offs[b0]), int(offs[b1])
    return offs[b0:b1 + 1] - lo, slice(lo, hi)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (the timed region's length)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(rows: np.ndarray, dst: int = 0):
    """Rank `dst` receives every rank's rows, concatenated in rank order (None elsewhere)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return rows
    out = [None] * dist.get_world_size() if dist.get_rank() == dst else None
    dist.gather_object(rows, out, dst=dst)
    if dist.get_rank() != dst:
        return None
    return np.concatenate([np.asarray(r).reshape(-1, *np.asarray(rows).shape[1:]) for r in out], axis=0)


# ---------------------------------------------------------------------------
# One very long series over several ranks: outer-index ranges with halos
# ---------------------------------------------------------------------------

def outer_ranges(n: int, world: int):
    """Contiguous index ranges [(j0, j1)] of n outer points, one per rank."""
    return [(n * r // world, n * (r + 1) // world) for r in range(world)]


def reach(lags, kernel: str, h: float, path: str = "auto", trunc_R: float = 0.0) -> float:
    """How far from an outer point s_j an inner point can still pair with it at any
    lag: max|tau| plus the kernel's half-width (h for the rectangle and Hann
    windows, R h for the windowed Gaussian, 10 h for the untruncated spectral
    Gaussian, whose weights beyond are below e^-50 of the peak), plus a margin
    for the rounding of the FP64 window bounds."""
    lags = np.asarray(lags, dtype=np.float64)
    if kernel in ("rectangle", "hanning"):
        w = h
    elif path == "windowed":
        w = (trunc_R if trunc_R > 0 else 8.0) * h
    else:
        w = 10.0 * h
    r = float(np.max(np.abs(lags))) + w
    return r * (1.0 + 1e-9) + 1e-6


def halo(t_inner, s_lo: float, s_hi: float, r: float):
    """Index range [i0, i1) of the sorted inner times within r of [s_lo, s_hi]."""
    t_inner = np.asarray(t_inner)
    return (int(np.searchsorted(t_inner, s_lo - r, side="left")),
            int(np.searchsorted(t_inner, s_hi + r, side="right")))


def pool(summaries):
    """(n, mean, std) of the union of point sets from their (n, mean, m2 = sum
    (x - mean)^2) summaries, combined pairwise in order (Chan, Golub, LeVeque)."""
    n, mean, m2 = 0, 0.0, 0.0
    for sm in summaries:
        nb, mb, m2b = int(sm["n"]), float(sm["mean"]), float(sm["m2"])
        if nb == 0:
            continue
        if n == 0:
            n, mean, m2 = nb, mb, m2b
            continue
        tot = n + nb
        d = mb - mean
        mean += d * nb / tot
        m2 += m2b + d * d * n * nb / tot
        n = tot
    if n == 0 or not m2 > 0.0:
        raise ValueError("the pooled series has zero variance: the standardised series is undefined")
    return {"n": n, "mean": mean, "std": float(np.sqrt(m2 / n))}


def _all_gather_objects(obj):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


def _all_reduce_sum(a: np.ndarray) -> np.ndarray:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return a
    t = torch.from_numpy(np.ascontiguousarray(a))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def split_series(t, x, lags, evaluate, summarize, rank=None, world=None, s=None, y=None, kernel="rectangle",
                 h=1.0, path="auto", trunc_R=0.0):
    """The ACF (s, y omitted) or CCF of one long series, split by outer index over
    `world` ranks (this call evaluates rank `rank`'s range; with a process group
    the ranks' partial sums are all-reduced, without one pass rank=None to run
    every range in turn and sum them here).

    summarize(t, x) -> dict(n, mean, m2) of a point set;
    evaluate(t_in, x_in, s_out, y_out, lags, acf, pooled) -> (num, den, count):
        the partial sums over the outer points (s_out, y_out) against the inner
        points (t_in, x_in) with the pooled standardisation, for the ACF (window
        centre s_j + tau, the whole series' convention) or the CCF (s_j - tau).

    Returns dict(c, b, count, num) of the whole series: c = N / max(B, 1e-16)."""
    t = np.asarray(t, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    lags = np.asarray(lags, dtype=np.float64)
    acf = s is None
    so = t if acf else np.asarray(s, dtype=np.float64)
    yo = x if acf else np.asarray(y, dtype=np.float64)
    if world is None:
        world = 1
    ranks = range(world) if rank is None else [rank]
    # pooled statistics: x over a partition of its own points, y over the outer ranges
    xparts = outer_ranges(t.size, world)
    oparts = outer_ranges(so.size, world)
    sx = [summarize(t[a:b], x[a:b]) for a, b in (xparts[r] for r in ranks)]
    sy = sx if acf else [summarize(so[a:b], yo[a:b]) for a, b in (oparts[r] for r in ranks)]
    gx = [g for part in _all_gather_objects(sx) for g in part] if rank is not None else sx
    gy = gx if acf else ([g for part in _all_gather_objects(sy) for g in part] if rank is not None else sy)
    px, py = pool(gx), pool(gy)
    pooled = {"mean_x": px["mean"], "std_x": px["std"], "n_x": px["n"],
              "mean_y": py["mean"], "std_y": py["std"], "n_y": py["n"]}
    r_ = reach(lags, kernel, h, path, trunc_R)
    K = lags.size
    num = np.zeros(K)
    den = np.zeros(K)
    cnt = np.zeros(K, dtype=np.int64)
    for r in ranks:
        j0, j1 = oparts[r]
        if j1 <= j0:
            continue
        i0, i1 = halo(t, so[j0], so[j1 - 1], r_)
        if i1 <= i0:
            continue
        n_, d_, c_ = evaluate(t[i0:i1], x[i0:i1], so[j0:j1], yo[j0:j1], lags, acf, pooled)
        num += n_
        den += d_
        cnt += np.asarray(c_, dtype=np.int64)
    if rank is not None:
        num = _all_reduce_sum(num)
        den = _all_reduce_sum(den)
        cnt = _all_reduce_sum(cnt)
    return {"c": num / np.maximum(den, 1e-16), "b": den, "count": cnt, "num": num}


def gpu_evaluator(api, kernel="rectangle", h=1.0, path="auto", precision="fp64", trunc_R=0.0, ctx=None):
    """evaluate() of split_series on the GPU library: the partial sums of one range
    through ncf_corr_pooled (inner halo as x at t, outer range as y at s; for an
    ACF the lags are negated, which puts the window centre at s_j + tau, the
    whole series' convention, with the same FP64 roundings)."""
    def evaluate(t_in, x_in, s_out, y_out, lags, acf, pooled):
        r = api.corr_pooled(t_in, x_in, -lags if acf else lags, pooled, kernel=kernel, h=h, s=s_out, y=y_out,
                            path=path, precision=precision, trunc_R=trunc_R, ctx=ctx)
        c = r["c"].cpu().numpy()
        b = r["b"].cpu().numpy()
        return c * np.maximum(b, 1e-16), b, r["count"].cpu().numpy()
    return evaluate


def gpu_summarizer(api, ctx=None):
    """summarize() of split_series on the GPU library (ncf_series_stats)."""
    def summarize(t, x):
        return api.series_stats(t, x, ctx=ctx)
    return summarize
