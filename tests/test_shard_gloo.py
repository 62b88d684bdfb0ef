"""The N > 1 path on CPU: world-size-2 gloo process groups run the series
partition, the per-rank evaluation (the oracle stands in for the GPU) and the
gather, and must reproduce the single-process result exactly."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
from paper_2609_03866_b300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    return synth.light_curves(B=7, n_lo=200, n_hi=1500, K=9, seed=synth.BASE_SEED + 3)


def _evaluate(w, b0, b1):
    rows = []
    for b in range(b0, b1):
        sl = slice(int(w.offs[b]), int(w.offs[b + 1]))
        r = oracle.corr(w.t[sl], w.x[sl], w.lags, "rectangle", 0.5, method="windowed")
        rows.append(np.concatenate([r["c"], r["count"].astype(np.float64)]))
    return np.asarray(rows, dtype=np.float64).reshape(b1 - b0, 2 * w.lags.size)


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert shard.dist_env()[:2] == (rank, world)
        w = _batch()
        b0, b1 = shard.partition_series(w.offs, w.lags.size, world)[rank]
        rows = shard.gather_rows(_evaluate(w, b0, b1))
        t_max = shard.max_over_ranks(1.0 + rank)
        dist.barrier()
        if rank == 0:
            np.savez(out_path, rows=rows, t_max=t_max)
    finally:
        dist.destroy_process_group()


def test_partition_covers_every_series_once():
    w = synth.light_curves(B=50, n_lo=200, n_hi=200_000, K=8)
    for world in (1, 2, 3, 8, 64):
        parts = shard.partition_series(w.offs, 256, world)
        assert parts[0][0] == 0 and parts[-1][1] == w.B and len(parts) == world
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        if world <= 8:
            cost = shard.series_cost(w.offs, 256)
            per = [cost[a:b].sum() for a, b in parts]
            assert max(per) <= cost.sum() / world + cost.max()   # within one series of even


def test_sub_batch_rebases_offsets():
    offs = np.array([0, 3, 10, 12, 20])
    o, sl = shard.sub_batch(offs, 1, 3)
    assert o.tolist() == [0, 7, 9] and (sl.start, sl.stop) == (3, 12)


def test_two_gloo_ranks_reproduce_one_process():
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "r.npz")
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
        got = np.load(out)
        w = _batch()
        ref = _evaluate(w, 0, w.B)
        assert np.array_equal(got["rows"], ref)
        assert float(got["t_max"]) == 2.0


# ---------------------------------------------------------------------------
# One long series split by outer index over world-size-2 gloo ranks; the oracle
# evaluates each rank's partial sums (the GPU version is test_gpu_split.py)
# ---------------------------------------------------------------------------

_KERN = {"gaussian": 0, "rectangle": 1}


def _oracle_summarize(t, x):
    m, sd = oracle.stats(x)
    return {"n": int(x.size), "mean": m, "m2": float(sd) ** 2 * x.size}


def _oracle_evaluator(kernel, h, trunc_R):
    def evaluate(t_in, x_in, s_out, y_out, lags, acf, pooled):
        xs = (np.asarray(x_in) - pooled["mean_x"]) / pooled["std_x"]
        ys = (np.asarray(y_out) - pooled["mean_y"]) / pooled["std_y"]
        return oracle._sums("windowed", np.ascontiguousarray(t_in), np.ascontiguousarray(xs),
                            np.ascontiguousarray(s_out), np.ascontiguousarray(ys), np.ascontiguousarray(lags),
                            _KERN[kernel], h, trunc_R, +1 if acf else -1)
    return evaluate


def _split_cases():
    w = synth.ou_ccf(nA=3000, nB=2400, K=23)
    a = synth.ar1_acf(n=2500, K=17)
    return [("acf", "rectangle", 1.0, 0.0, a.t, a.x, None, None, a.lags),
            ("acf", "gaussian", 1.0, 8.0, a.t, a.x, None, None, a.lags),
            ("ccf", "rectangle", 0.5, 0.0, w.t, w.x, w.s, w.y, w.lags),
            ("ccf", "gaussian", 0.5, 8.0, w.t, w.x, w.s, w.y, w.lags)]


def _split_worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        for i, (_, kernel, h, R, t, x, s, y, lags) in enumerate(_split_cases()):
            r = shard.split_series(t, x, lags, _oracle_evaluator(kernel, h, R), _oracle_summarize, rank=rank,
                                   world=world, s=s, y=y, kernel=kernel, h=h, path="windowed", trunc_R=R)
            res[f"c{i}"], res[f"n{i}"] = r["c"], r["count"]
        dist.barrier()
        if rank == 0:
            np.savez(out_path, **res)
    finally:
        dist.destroy_process_group()


def test_pool_matches_the_whole_series_statistics():
    rng = np.random.default_rng(9)
    x = rng.normal(size=10001) * 3.0 + 1e4
    parts = [x[:17], x[17:5000], x[5000:5001], x[5001:]]
    p = shard.pool([_oracle_summarize(None, v) for v in parts])
    m, sd = oracle.stats(x)
    assert p["n"] == x.size and abs(p["mean"] - m) < 1e-11 * abs(m) and abs(p["std"] / sd - 1) < 1e-12


def test_halo_covers_every_pair_of_a_range():
    t = np.sort(np.random.default_rng(4).uniform(0, 100, 400))
    lags = np.array([-7.0, 0.0, 3.5])
    r = shard.reach(lags, "rectangle", 0.5)
    for j0, j1 in shard.outer_ranges(t.size, 5):
        i0, i1 = shard.halo(t, t[j0], t[j1 - 1], r)
        inside = (t >= t[j0] - 7.5) & (t <= t[j1 - 1] + 7.5)
        assert np.all(np.flatnonzero(inside) >= i0) and np.all(np.flatnonzero(inside) < i1)


def test_two_gloo_ranks_split_one_series_exactly():
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "s.npz")
        mp.start_processes(_split_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
        got = np.load(out)
        for i, (kind, kernel, h, R, t, x, s, y, lags) in enumerate(_split_cases()):
            ref = oracle.corr(t, x, lags, kernel, h, s=s, y=y, method="windowed", trunc_R=R)
            assert np.array_equal(got[f"n{i}"], ref["count"]), (kind, kernel)
            assert np.max(np.abs(got[f"c{i}"] - ref["c"])) < 1e-12, (kind, kernel)
