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
TOL = {lp2d.PREC_FP32: 1e-4, lp2d.PREC_FP32_F64ISECT: 1e-4, lp2d.PREC_FP64: 1e-10}  # as the parity tests


def _to_dev(batch):
    return {k: torch.from_numpy(np.ascontiguousarray(batch[k])).to(DEV) for k in ("ax", "ay", "b", "offsets", "obj")}


def _solve(batch, entry, precision, schedule):
    t = _to_dev(batch)
    n_lp = len(batch["offsets"]) - 1
    opts = lp2d.default_options(precision=precision, schedule=schedule)
    dtype = torch.float64 if precision == lp2d.PREC_FP64 else torch.float32
    xy = torch.full((2 * n_lp,), 12345.0, dtype=dtype, device=DEV)
    st = torch.full((n_lp,), -9, dtype=torch.int32, device=DEV)
    if entry == "noalloc":
        lp2d.solve_batch_noalloc(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"], xy, st,
                                 opts)
    else:  # the existing entry point, with a workspace of its own
        lp2d.solve_batch_ex(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"], xy, st,
                            opts, lp2d.new_workspace(n_lp, opts, device=DEV))
    torch.cuda.synchronize()
    return xy.cpu().numpy().reshape(-1, 2).astype(np.float64), st.cpu().numpy()


def _compare(batch, got, ref, tol):
    (gxy, gst), (rxy, rst) = got, ref
    assert (gst == rst).all()
    c = batch["obj"].astype(np.float64)
    solved = (rst == lp2d.OPTIMAL) | (rst == lp2d.BOX_BOUNDED)
    f_got = np.einsum("ij,ij->i", gxy, c)[solved]
    f_ref = np.einsum("ij,ij->i", rxy, c)[solved]
    assert (np.abs(f_got - f_ref) / np.maximum(np.abs(f_ref), 1.0)).max(initial=0.0) <= tol
    assert np.isnan(gxy[~solved]).all()


@pytest.mark.parametrize("precision,schedule", [
    (lp2d.PREC_FP32, lp2d.SCHED_PERSISTENT), (lp2d.PREC_FP32_F64ISECT, lp2d.SCHED_PERSISTENT),
    (lp2d.PREC_FP64, lp2d.SCHED_PERSISTENT), (lp2d.PREC_FP32, lp2d.SCHED_UNIFORM),
    (lp2d.PREC_FP64, lp2d.SCHED_UNIFORM)])
def test_noalloc_matches_allocating_entry_point_on_two_calls_in_a_row(precision, schedule):
    # Two different batches, one call each, back to back: the second call finds the
    # first call's leftovers in the shared scratch array.  Sizes cover the per-warp,
    # per-team and read-through-HBM paths.
    sizes = workloads.loguniform_sizes(np.random.default_rng(3), 6000, 8, 3000)
    first = workloads.disk_batch(sizes, seed=31, infeasible_frac=0.1)
    second = workloads.plain_at_scale(seed=32, n_lp=5000)
    got1 = _solve(first, "noalloc", precision, schedule)
    got2 = _solve(second, "noalloc", precision, schedule)
    _compare(first, got1, _solve(first, "existing", precision, schedule), TOL[precision])
    _compare(second, got2, _solve(second, "existing", precision, schedule), TOL[precision])
