"""Multi-rank host logic on CPU: two gloo ranks shard a batch (2-D, and 5-D for the
d-dimensional solver's layout), solve their ranges with the oracle, and together
reproduce the single-process result."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1902_04995_gb300 import dist as lpdist  # noqa: E402
from paper_1902_04995_gb300 import workloads  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_partition_and_balance():
    batch = workloads.ragged(n_lp=5000)
    off = batch["offsets"]
    for world in (1, 2, 3, 8):
        ranges = [lpdist.shard_lp_range(off, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == 5000
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        work = [off[h] - off[l] for l, h in ranges]
        assert max(work) - min(work) <= 2 * 2049  # within a couple of LPs of equal
    with pytest.raises(ValueError):
        lpdist.shard_lp_range(off, 2, 2)


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle

        batch = workloads.ragged(n_lp=3000, seed=11)
        lo, hi = lpdist.shard_lp_range(batch["offsets"], rank, world)
        sub, sub_seed = lpdist.slice_batch(batch, lo, hi, seed=7)
        res = oracle.solve_batch(sub["ax"], sub["ay"], sub["b"], sub["offsets"], sub["obj"], sub["box"],
                                 seed=sub_seed, want_nviol=True)
        # gather every rank's piece on every rank
        pieces = [None] * world
        dist.all_gather_object(pieces, (lo, hi, res["status"], res["xy"], res["nviol"]))
        slowest = lpdist.max_over_ranks(float(rank + 1))
        dist.barrier()
        if rank == 0:
            np.save(os.path.join(out_dir, "slowest.npy"), np.array([slowest]))
            st = np.concatenate([p[2] for p in sorted(pieces, key=lambda p: p[0])])
            xy = np.concatenate([p[3] for p in sorted(pieces, key=lambda p: p[0])])
            nv = np.concatenate([p[4] for p in sorted(pieces, key=lambda p: p[0])])
            np.savez(os.path.join(out_dir, "merged.npz"), st=st, xy=xy, nv=nv)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_single_process_result(tmp_path, oracle_mod):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    merged = np.load(tmp_path / "merged.npz")
    assert float(np.load(tmp_path / "slowest.npy")[0]) == 2.0
    batch = workloads.ragged(n_lp=3000, seed=11)
    ref = oracle_mod.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"], batch["box"],
                                 seed=7, want_nviol=True)
    assert (merged["st"] == ref["status"]).all()
    assert (merged["nv"] == ref["nviol"]).all()  # same visit orders: seeds follow the global LP index
    assert np.array_equal(merged["xy"], ref["xy"], equal_nan=True)


def _rank_main_nd(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle

        batch = workloads.ball_batch(5, workloads.loguniform_sizes(np.random.default_rng(3), 300, 4, 200), seed=12,
                                     infeasible_frac=0.1)
        lo, hi = lpdist.shard_lp_range(batch["offsets"], rank, world)
        sub, sub_seed = lpdist.slice_batch(batch, lo, hi, seed=5)
        assert sub["a"].shape == (5, int(sub["offsets"][-1]))
        res = oracle.solve_batchN(sub["a"], sub["b"], sub["offsets"], sub["obj"], sub["box"], seed=sub_seed,
                                  want_nviol=True)
        pieces = [None] * world
        dist.all_gather_object(pieces, (lo, res["status"], res["x"], res["nviol"]))
        dist.barrier()
        if rank == 0:
            pieces.sort(key=lambda p: p[0])
            np.savez(os.path.join(out_dir, "merged_nd.npz"), st=np.concatenate([p[1] for p in pieces]),
                     x=np.concatenate([p[2] for p in pieces]), nv=np.concatenate([p[3] for p in pieces]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_a_5d_batch(tmp_path, oracle_mod):
    world = 2
    mp.spawn(_rank_main_nd, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    merged = np.load(tmp_path / "merged_nd.npz")
    batch = workloads.ball_batch(5, workloads.loguniform_sizes(np.random.default_rng(3), 300, 4, 200), seed=12,
                                 infeasible_frac=0.1)
    ref = oracle_mod.solve_batchN(batch["a"], batch["b"], batch["offsets"], batch["obj"], batch["box"], seed=5,
                                  want_nviol=True)
    assert (merged["st"] == ref["status"]).all()
    assert (merged["nv"] == ref["nviol"]).all()
    assert np.array_equal(merged["x"], ref["x"], equal_nan=True)


def test_max_over_ranks_without_process_group():
    assert lpdist.max_over_ranks(3.5) == 3.5
