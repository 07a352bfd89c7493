"""lp2d_solve_batch_noalloc, the entry point for callers that cannot allocate device
memory (its queue scratch is a fixed device array inside the library), must give
the same results as the allocating entry point.

Collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1902_04995_gb300 import lp2d, workloads  # noqa: E402

DEV = torch.device("cuda:0")
TOL = 1e-4  # the FP32 objective tolerance of the parity tests


def _to_dev(batch):
    return {k: torch.from_numpy(np.ascontiguousarray(batch[k])).to(DEV) for k in ("ax", "ay", "b", "offsets", "obj")}


def _solve(batch, entry):
    t = _to_dev(batch)
    n_lp = len(batch["offsets"]) - 1
    xy = torch.full((2 * n_lp,), 12345.0, dtype=torch.float32, device=DEV)
    st = torch.full((n_lp,), -9, dtype=torch.int32, device=DEV)
    if entry == "noalloc":
        lp2d.solve_batch_noalloc(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"], xy, st)
    else:
        lp2d.solve_batch(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"], xy, st)
    torch.cuda.synchronize()
    return xy.cpu().numpy().reshape(-1, 2).astype(np.float64), st.cpu().numpy()


def _compare(batch, got, ref):
    (gxy, gst), (rxy, rst) = got, ref
    assert (gst == rst).all()
    c = batch["obj"].astype(np.float64)
    solved = (rst == lp2d.OPTIMAL) | (rst == lp2d.BOX_BOUNDED)
    f_got = np.einsum("ij,ij->i", gxy, c)[solved]
    f_ref = np.einsum("ij,ij->i", rxy, c)[solved]
    assert (np.abs(f_got - f_ref) / np.maximum(np.abs(f_ref), 1.0)).max(initial=0.0) <= TOL
    assert np.isnan(gxy[~solved]).all()


def test_noalloc_matches_allocating_entry_point_on_two_calls_in_a_row():
    # Two different batches, one call each, back to back: the second call finds the
    # first call's leftovers in the shared scratch array.  Sizes cover the per-warp,
    # per-team and read-through-HBM paths.
    sizes = workloads.loguniform_sizes(np.random.default_rng(3), 6000, 8, 3000)
    first = workloads.disk_batch(sizes, seed=31, infeasible_frac=0.1)
    second = workloads.plain_at_scale(seed=32, n_lp=5000)
    got1 = _solve(first, "noalloc")
    got2 = _solve(second, "noalloc")
    _compare(first, got1, _solve(first, "existing"))
    _compare(second, got2, _solve(second, "existing"))
