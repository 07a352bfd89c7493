"""Host-side helpers for running the solver with one process per GPU.

LPs are independent, so a batch shards with no exchange step: rank r solves a
contiguous range of LPs and writes its own slice of the results.  Ranges are cut so
that every rank gets about the same number of constraints (the work is linear in
it: expected O(m) per LP for Seidel's method with a random order, Sec. 2.1).

The visit order of LP l is seeded with seed + l, where l is the LP's index in the
whole batch; a rank solving LPs lo..hi-1 therefore passes seed + lo, so each LP's
result does not depend on how the batch was split.

The only collectives are for measurement: a barrier and a max over ranks of the
step time.
"""
from __future__ import annotations

import numpy as np


def shard_lp_range(offsets, rank: int, world: int):
    """Contiguous LP range [lo, hi) of `rank` out of `world`, with about equal
    constraint counts.  offsets: int64 CSR offsets of the whole batch."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} out of range for world size {world}")
    offsets = np.asarray(offsets, dtype=np.int64)
    n_lp = offsets.shape[0] - 1
    total = offsets[-1] - offsets[0]

    def cut(r):
        if r <= 0:
            return 0
        if r >= world:
            return n_lp
        target = offsets[0] + (total * r) // world
        return int(np.searchsorted(offsets, target, side="left").clip(0, n_lp))

    return cut(rank), cut(rank + 1)


def slice_batch(batch, lo: int, hi: int, seed: int = 0):
    """LPs lo..hi-1 of a batch as a batch of their own (views into the arrays,
    offsets rebased to 0), and the seed that keeps their visit orders unchanged.
    Works for 2-D (ax, ay, b), 3-D (ax, ay, az, b) and d-dimensional (a [d, n], b)
    batches."""
    off = batch["offsets"]
    s, e = int(off[lo]), int(off[hi])
    sub = dict(batch)
    for key in ("ax", "ay", "az", "b"):
        if key in batch:
            sub[key] = batch[key][s:e]
    if "a" in batch:
        sub["a"] = batch["a"][:, s:e]
    sub.update({"offsets": off[lo:hi + 1] - s, "obj": batch["obj"][lo:hi]})
    if "infeasible" in batch:
        sub["infeasible"] = batch["infeasible"][lo:hi]
    return sub, seed + lo


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks of the default process group (the value
    itself when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
