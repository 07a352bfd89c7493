"""lp2d_solve_batch_host: the host-buffer entry point that copies the batch in chunks
and overlaps each chunk's copy with the previous chunk's solve.  Its results must
equal those of one device-resident lp2d_solve_batch_ex call over the whole batch
(every LP keeps its seed, seed + l), and match the FP64 oracle."""
from __future__ import annotations

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1902_04995_gb300 import lp2d, workloads  # noqa: E402

DEV = torch.device("cuda:0")
THREADS = os.cpu_count() or 1


def host_tensors(batch, pinned=True):
    out = {}
    for k in ("ax", "ay", "b", "offsets", "obj"):
        t = torch.from_numpy(np.ascontiguousarray(batch[k]).reshape(-1))
        out[k] = t.pin_memory() if pinned else t.clone()
    return out


def host_solve(batch, seed=0, precision=lp2d.PREC_FP32, pinned=True):
    h = host_tensors(batch, pinned)
    n_lp = h["offsets"].numel() - 1
    dt = torch.float64 if precision == lp2d.PREC_FP64 else torch.float32
    xy = torch.full((2 * n_lp,), 12345.0, dtype=dt)
    st = torch.full((n_lp,), -9, dtype=torch.int32)
    if pinned:
        xy, st = xy.pin_memory(), st.pin_memory()
    opts = lp2d.default_options(seed=seed, precision=precision)
    lp2d.solve_batch_host(h["ax"], h["ay"], h["b"], h["offsets"], h["obj"], batch["box"], xy, st, opts)
    torch.cuda.current_stream().synchronize()
    return xy.numpy().reshape(-1, 2).copy(), st.numpy().copy()


def device_solve(batch, seed=0, precision=lp2d.PREC_FP32):
    t = {k: torch.from_numpy(np.ascontiguousarray(batch[k]).reshape(-1)).to(DEV)
         for k in ("ax", "ay", "b", "offsets", "obj")}
    n_lp = t["offsets"].numel() - 1
    dt = torch.float64 if precision == lp2d.PREC_FP64 else torch.float32
    xy = torch.empty(2 * n_lp, dtype=dt, device=DEV)
    st = torch.empty(n_lp, dtype=torch.int32, device=DEV)
    opts = lp2d.default_options(seed=seed, precision=precision)
    lp2d.solve_batch_ex(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"], batch["box"], xy, st, opts,
                        lp2d.new_workspace(n_lp, opts, device=DEV))
    torch.cuda.synchronize()
    return xy.cpu().numpy().reshape(-1, 2), st.cpu().numpy()


def assert_same(a, b):
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[0], b[0], equal_nan=True)


def test_chunked_ragged_batch_equals_one_device_call():
    # about 48M constraints: five chunks of decreasing size, both device slots reused
    batch = workloads.ragged(n_lp=131072)
    assert batch["offsets"][-1] > 8 * (4 << 20)
    assert_same(host_solve(batch, seed=3), device_solve(batch, seed=3))


@pytest.mark.parametrize("precision", [lp2d.PREC_FP32, lp2d.PREC_FP32_F64ISECT, lp2d.PREC_FP64])
def test_precisions_equal_device_call_on_collision_workload(precision):
    batch = workloads.collision()
    assert_same(host_solve(batch, seed=1, precision=precision), device_solve(batch, seed=1, precision=precision))


def test_small_batch_matches_the_oracle():
    batch = workloads.plain_small()
    xy, st = host_solve(batch, seed=5)
    ref = oracle.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"], batch["box"],
                             seed=5, threads=THREADS)
    assert np.array_equal(st, ref["status"])
    ok = ref["status"] != oracle.INFEASIBLE
    c = batch["obj"].astype(np.float64)
    f_ref = (c * ref["xy"]).sum(1)
    f_got = (c * xy.astype(np.float64)).sum(1)
    rel = np.abs(f_got - f_ref)[ok] / np.maximum(np.abs(f_ref[ok]), 1.0)
    assert rel.max(initial=0.0) <= 1e-4
    assert np.isnan(xy[~ok]).all()


def test_pageable_memory_and_nonzero_first_offset():
    batch = workloads.ragged(n_lp=4000, seed=2)
    # drop the first 10 LPs but keep the constraint arrays whole: offsets start above 0
    cut = dict(batch)
    cut["offsets"] = batch["offsets"][10:]
    cut["obj"] = batch["obj"][10:]
    got = host_solve(cut, seed=10, pinned=False)
    ref = device_solve(batch, seed=0)
    assert np.array_equal(got[1], ref[1][10:])
    assert np.array_equal(got[0], ref[0][10:], equal_nan=True)


def test_growing_and_shrinking_calls_and_empty_batch():
    small = workloads.plain_small()
    big = workloads.ragged(n_lp=40000, seed=4)
    for b in (small, big, small):
        assert_same(host_solve(b, seed=2), device_solve(b, seed=2))
    empty = {"ax": np.zeros(0, np.float32), "ay": np.zeros(0, np.float32), "b": np.zeros(0, np.float32),
             "offsets": np.zeros(1, np.int64), "obj": np.zeros((0, 2), np.float32), "box": small["box"]}
    xy, st = host_solve(empty)
    assert xy.size == 0 and st.size == 0
