"""Error of each precision mode against the FP64 oracle on the collision-avoidance
workload (16,384 LPs: a 16-gon speed limit plus 10-100 neighbour half-planes, 5 % of
them within 1e-6 rad of an earlier normal), with the GPU time of one solve.

    python tests/precision_report.py [--seed S]

Prints one JSON line per mode.  Needs a CUDA device and the built library."""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import oracle  # noqa: E402
from paper_1902_04995_gb300 import lp2d, workloads  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workload", default="collision_16384", choices=sorted(workloads.WORKLOADS))
    args = ap.parse_args()
    batch = workloads.WORKLOADS[args.workload]()
    ref = oracle.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"], batch["box"],
                             seed=args.seed, threads=os.cpu_count() or 1)
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(np.ascontiguousarray(batch[k])).to(dev) for k in ("ax", "ay", "b", "offsets", "obj")}
    n_lp = len(batch["offsets"]) - 1
    c = batch["obj"].astype(np.float64)
    off = batch["offsets"]
    owner = np.repeat(np.arange(n_lp), np.diff(off))
    for name, prec in (("fp32", lp2d.PREC_FP32), ("fp32_f64isect", lp2d.PREC_FP32_F64ISECT),
                       ("fp64", lp2d.PREC_FP64)):
        solver = lp2d.Solver(n_lp, lp2d.default_options(seed=args.seed, precision=prec), device=dev)
        solver(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            solver(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"])
        e1.record()
        torch.cuda.synchronize()
        xy = solver.out_xy.cpu().numpy().reshape(-1, 2).astype(np.float64)
        st = solver.out_status.cpu().numpy()
        both = (st != oracle.INFEASIBLE) & (ref["status"] != oracle.INFEASIBLE) & (st != oracle.BAD_INPUT)
        f = np.einsum("ij,ij->i", xy, c)
        fr = np.einsum("ij,ij->i", ref["xy"], c)
        rel = np.abs(f - fr)[both] / np.maximum(np.abs(fr[both]), 1.0)
        # largest violation of any constraint by the returned point, relative to max(1, |x|)
        slack = batch["ax"] * xy[owner, 0] + batch["ay"] * xy[owner, 1] - batch["b"]
        scale = np.maximum(1.0, np.abs(xy[owner]).max(axis=1))
        viol = np.where(both[owner], slack / scale, -np.inf)
        print(json.dumps({
            "workload": args.workload, "mode": name, "ms_per_solve": e0.elapsed_time(e1) / 10,
            "status_mismatches": int((st != ref["status"]).sum()), "n_lp": n_lp,
            "max_rel_objective_error": float(rel.max(initial=0.0)),
            "p99_rel_objective_error": float(np.percentile(rel, 99)) if rel.size else 0.0,
            "max_rel_constraint_violation": float(max(viol.max(initial=-np.inf), 0.0)),
        }), flush=True)


if __name__ == "__main__":
    main()
