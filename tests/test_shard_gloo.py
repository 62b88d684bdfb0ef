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
