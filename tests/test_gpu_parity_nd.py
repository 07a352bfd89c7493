"""GPU parity of the batched d-dimensional solver (lpnd_solve_batch, d = 2..5) against
the FP64 d-dimensional oracle on the same seeded inputs: status bit-exact, the
objective within 1e-4 relative (FP32) or 1e-10 (FP64) of max(|f_oracle|, 1); in FP64
also the number of violations and the d defining constraints.  At 65,536 LPs the
oracle solves a seeded sample one LP at a time, and every LP is checked against what
holds at any size: infeasible exactly where the generator made it so, and every
returned vertex inside the box and every constraint."""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

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
TOL = {lp2d.PREC_FP32: 1e-4, lp2d.PREC_FP64: 1e-10}


def gpu_solve_nd(batch, seed=0, precision=lp2d.PREC_FP32, want=False, **tune):
    d = batch["a"].shape[0]
    a = torch.from_numpy(np.ascontiguousarray(batch["a"])).to(DEV)
    b = torch.from_numpy(batch["b"]).to(DEV)
    off = torch.from_numpy(batch["offsets"]).to(DEV)
    obj = torch.from_numpy(np.ascontiguousarray(batch["obj"]).reshape(-1)).to(DEV)
    n_lp = len(batch["offsets"]) - 1
    nviol = torch.full((max(n_lp, 1),), -7, dtype=torch.int32, device=DEV) if want else None
    dfn = torch.full((max(d * n_lp, 1),), -7, dtype=torch.int32, device=DEV) if want else None
    opts = lp2d.default_options(seed=seed, precision=precision, out_nviol=nviol.data_ptr() if want else None,
                                out_def=dfn.data_ptr() if want else None, **tune)
    dt = torch.float64 if precision == lp2d.PREC_FP64 else torch.float32
    x = torch.full((max(d * n_lp, 1),), 12345.0, dtype=dt, device=DEV)
    st = torch.full((max(n_lp, 1),), -9, dtype=torch.int32, device=DEV)
    ws = lp2d.new_workspace(n_lp, opts, device=DEV)
    lp2d.solve_batch_nd(a, b, off, obj, batch["box"], x, st, opts, ws)
    torch.cuda.synchronize()
    res = {"x": x[:d * n_lp].cpu().numpy().reshape(-1, d).astype(np.float64), "status": st[:n_lp].cpu().numpy(),
           "err": lp2d.read_device_error(ws)}
    if want:
        res["nviol"] = nviol[:n_lp].cpu().numpy()
        res["def"] = dfn[:d * n_lp].cpu().numpy().reshape(-1, d)
    return res


def oracle_nd(batch, seed=0, **kw):
    return oracle.solve_batchN(batch["a"], batch["b"], batch["offsets"], batch["obj"], batch["box"], seed=seed,
                               threads=THREADS, **kw)


def oracle_sample(batch, lps, seed=0):
    """The oracle on LPs `lps` of the batch, each with its own seed (seed + l)."""
    d = batch["a"].shape[0]

    def one(l):
        s, e = batch["offsets"][l], batch["offsets"][l + 1]
        r = oracle.solve_batchN(batch["a"][:, s:e], batch["b"][s:e], np.array([0, e - s]), batch["obj"][l:l + 1],
                                batch["box"], seed=seed + int(l))
        return r["x"][0], r["status"][0]

    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        out = list(ex.map(one, lps))
    return {"x": np.array([o[0] for o in out]).reshape(-1, d), "status": np.array([o[1] for o in out], np.int32)}


def assert_parity(obj, got, ref, tol):
    bad = np.nonzero(got["status"] != ref["status"])[0]
    assert bad.size == 0, (f"{bad.size} status mismatches, first {bad[:8]}: gpu {got['status'][bad[:8]]} "
                           f"oracle {ref['status'][bad[:8]]}")
    c = obj.astype(np.float64)
    solved = (ref["status"] == oracle.OPTIMAL) | (ref["status"] == oracle.BOX_BOUNDED)
    f_ref = np.einsum("ij,ij->i", ref["x"], c)[solved]
    f_got = np.einsum("ij,ij->i", got["x"], c)[solved]
    err = np.abs(f_got - f_ref) / np.maximum(np.abs(f_ref), 1.0)
    assert err.size == 0 or err.max() <= tol, f"max rel objective error {err.max():.3e}"
    assert np.isnan(got["x"][~solved]).all()
    return err.max(initial=0.0)


def assert_primal_feasible(batch, got, slack=1e-4):
    """Every returned vertex satisfies the box and every constraint of its LP within
    `slack` relative to the terms of the constraint."""
    d = batch["a"].shape[0]
    ok = got["status"] != oracle.INFEASIBLE
    owner = np.repeat(np.arange(len(batch["offsets"]) - 1), np.diff(batch["offsets"]))
    keep = ok[owner]
    x = got["x"][owner[keep]]
    a = batch["a"][:, keep].T.astype(np.float64)
    b = batch["b"][keep].astype(np.float64)
    lhs = np.einsum("ij,ij->i", a, x)
    assert (lhs - b <= slack * (np.abs(a * x).sum(1) + np.abs(b) + 1.0)).all()
    lo = np.array(batch["box"][0::2]) - slack * 1e3
    hi = np.array(batch["box"][1::2]) + slack * 1e3
    assert ((got["x"][ok] >= lo) & (got["x"][ok] <= hi)).all()
    assert got["x"][ok].shape[1] == d


@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP64])
@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_small_batches_match_the_oracle(d, prec):
    cap = lp2d.warp_stage_constraints_nd(d)
    n_rag = 1000 if d < 5 else 400
    for sizes, seed in ((np.full(400, 40), 1), (workloads.loguniform_sizes(np.random.default_rng(d), n_rag, 1, cap - 1), 2)):
        batch = workloads.ball_batch(d, sizes, seed=seed + 10 * d, infeasible_frac=0.1)
        assert_parity(batch["obj"], gpu_solve_nd(batch, seed=3, precision=prec), oracle_nd(batch, seed=3), TOL[prec])


@pytest.mark.parametrize("d", [3, 4, 5])
def test_fp64_violation_counts_and_defining_planes_match_the_oracle(d):
    sizes = workloads.loguniform_sizes(np.random.default_rng(6 + d), 600, 1, lp2d.warp_stage_constraints_nd(d) - 1)
    batch = workloads.ball_batch(d, sizes, seed=4, infeasible_frac=0.1)
    got = gpu_solve_nd(batch, seed=5, precision=lp2d.PREC_FP64, want=True)
    ref = oracle_nd(batch, seed=5, want_def=True, want_nviol=True)
    assert_parity(batch["obj"], got, ref, TOL[lp2d.PREC_FP64])
    # the same FP64 steps in the same order, ties included (R23, R24): the oracle's path
    assert (got["nviol"] == ref["nviol"]).all()
    ok = ref["status"] != oracle.INFEASIBLE
    assert (np.sort(got["def"][ok], 1) == np.sort(ref["def"][ok], 1)).all()
    assert (got["def"][~ok] == np.iinfo(np.int32).min).all()


@pytest.mark.parametrize("d", [4, 5])
def test_ragged_at_scale(d):
    batch = workloads.ragged_nd(d)
    got = gpu_solve_nd(batch, seed=0)
    assert got["err"] == 0
    # at any size: infeasible exactly where the generator made it so, every vertex feasible
    assert np.array_equal(got["status"] == oracle.INFEASIBLE, batch["infeasible"])
    assert_primal_feasible(batch, got)
    # a seeded sample against the oracle, the largest LPs included
    n_lp = len(batch["offsets"]) - 1
    sizes = np.diff(batch["offsets"])
    rng = np.random.default_rng(d)
    lps = np.unique(np.r_[rng.choice(n_lp, 1200 if d == 4 else 600, replace=False), np.argsort(-sizes)[:16],
                          n_lp - 1])
    ref = oracle_sample(batch, lps, seed=0)
    assert_parity(batch["obj"][lps], {"x": got["x"][lps], "status": got["status"][lps]}, ref, TOL[lp2d.PREC_FP32])


@pytest.mark.parametrize("d", [2, 4, 5])
def test_edge_cases_empty_tiny_bad_and_too_large(d):
    cap = lp2d.max_constraints_nd(d)
    small = 512 - 2 * d
    half = lp2d.warp_stage_constraints_nd(d)
    # the quarter- and half-stage boundaries, the large-LP kernel up to its cap, and
    # one LP above the cap
    sizes = np.array([0, 1, 2, d, 2 * d - 1, 2 * d, 31, 32, 33, small - 1, small, small + 1, half - 1, half, half + 1,
                      5000, cap - 1, cap, cap + 1])
    batch = workloads.ball_batch(d, sizes, seed=7)
    got = gpu_solve_nd(batch, seed=1)
    keep = sizes <= cap
    assert (got["status"][~keep] == oracle.BAD_INPUT).all() and np.isnan(got["x"][~keep]).all()
    assert got["err"] & lp2d.DEVERR_TOO_LARGE
    sub = {k: (v[:, :int(batch["offsets"][keep.sum()])] if k == "a" else v) for k, v in batch.items()}
    sub["b"] = batch["b"][:int(batch["offsets"][keep.sum()])]
    sub["offsets"] = batch["offsets"][:keep.sum() + 1]
    sub["obj"] = batch["obj"][keep]
    ref = oracle_nd(sub, seed=1)
    assert_parity(sub["obj"], {"x": got["x"][keep], "status": got["status"][keep]}, ref, TOL[lp2d.PREC_FP32])
    # no constraints: the box corner, box-bounded
    assert got["status"][0] == oracle.BOX_BOUNDED
    assert np.array_equal(got["x"][0], np.where(batch["obj"][0] >= 0, 1e3, -1e3))
    # NaN data and a reversed LP (negative size) are BAD_INPUT
    b2 = workloads.ball_batch(d, np.array([10, 10, 10]), seed=8)
    b2["a"][d - 1, 12] = np.nan
    got = gpu_solve_nd(b2)
    assert got["status"][1] == oracle.BAD_INPUT and got["status"][0] != oracle.BAD_INPUT
    assert got["status"][2] != oracle.BAD_INPUT
    b2["offsets"] = np.array([0, 10, 5, 30], np.int64)
    got = gpu_solve_nd(b2)
    assert got["status"][1] == oracle.BAD_INPUT and got["err"] & lp2d.DEVERR_BAD_OFFSETS


def test_results_identical_across_tuning_and_repeated_launches():
    d = 4
    batch = workloads.ball_batch(d, workloads.loguniform_sizes(np.random.default_rng(3), 5000, 4, 1000), seed=9,
                                 infeasible_frac=0.1)
    base = gpu_solve_nd(batch, seed=2)
    for tune in ({"chunk_small": 1}, {"chunk_small": 16, "ctas_per_sm": 1}):
        got = gpu_solve_nd(batch, seed=2, **tune)
        assert (got["status"] == base["status"]).all()
        assert np.array_equal(got["x"], base["x"], equal_nan=True)
    # the workspace is reused without a memset
    a = torch.from_numpy(batch["a"]).to(DEV)
    b = torch.from_numpy(batch["b"]).to(DEV)
    off = torch.from_numpy(batch["offsets"]).to(DEV)
    obj = torch.from_numpy(batch["obj"].reshape(-1)).to(DEV)
    n = len(batch["offsets"]) - 1
    opts = lp2d.default_options(seed=2)
    ws = lp2d.new_workspace(n, opts, device=DEV)
    x = torch.empty(d * n, device=DEV)
    st = torch.empty(n, dtype=torch.int32, device=DEV)
    for _ in range(3):
        lp2d.solve_batch_nd(a, b, off, obj, batch["box"], x, st, opts, ws)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == base["status"]).all()
    assert np.array_equal(x.cpu().numpy().reshape(-1, d).astype(np.float64), base["x"], equal_nan=True)


@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP64])
@pytest.mark.parametrize("d", [4, 5])
def test_degenerate_lifted_lps_match_the_oracle(d, prec):
    # a (d-1)-dimensional batch with a zero last coefficient and a zero last objective
    # entry: every optimum is a segment along the last axis (BOX_BOUNDED on both sides),
    # box-vertex candidates are singular, and the objective must still match
    low = workloads.ball_batch(d - 1, workloads.loguniform_sizes(np.random.default_rng(40 + d), 600, 1, 500),
                               seed=41 + d, infeasible_frac=0.15)
    n = low["a"].shape[1]
    batch = {"a": np.vstack([low["a"], np.zeros((1, n), np.float32)]), "b": low["b"], "offsets": low["offsets"],
             "obj": np.hstack([low["obj"], np.zeros((600, 1), np.float32)]),
             "box": tuple(low["box"]) + (-7.0, 3.0)}
    got = gpu_solve_nd(batch, seed=4, precision=prec)
    ref = oracle_nd(batch, seed=4)
    assert_parity(batch["obj"], got, ref, TOL[prec])
    assert (got["status"][ref["status"] != oracle.INFEASIBLE] == oracle.BOX_BOUNDED).all()


@pytest.mark.parametrize("d", [3, 4, 5])
def test_duplicate_and_zero_normal_constraints_match_the_oracle(d):
    rng = np.random.default_rng(50 + d)
    base = workloads.ball_batch(d, np.full(300, 60), seed=51 + d, infeasible_frac=0.1)
    a_parts, b_parts, sizes = [], [], []
    for l in range(300):
        s, e = base["offsets"][l], base["offsets"][l + 1]
        a, b = base["a"][:, s:e], base["b"][s:e]
        dup = rng.choice(e - s, size=10)  # exact copies of ten of its constraints
        zero_b = np.where(np.arange(3) < 2, 1.0, -1.0 if l % 7 == 0 else 2.0).astype(np.float32)
        a = np.hstack([a, a[:, dup], np.zeros((d, 3), np.float32)])
        b = np.r_[b, b[dup], zero_b].astype(np.float32)
        perm = rng.permutation(a.shape[1])
        a_parts.append(a[:, perm])
        b_parts.append(b[perm])
        sizes.append(a.shape[1])
    offsets = np.zeros(301, np.int64)
    np.cumsum(sizes, out=offsets[1:])
    batch = {"a": np.ascontiguousarray(np.hstack(a_parts)), "b": np.concatenate(b_parts), "offsets": offsets,
             "obj": base["obj"], "box": base["box"]}
    for prec in (lp2d.PREC_FP32, lp2d.PREC_FP64):
        got = gpu_solve_nd(batch, seed=6, precision=prec)
        ref = oracle_nd(batch, seed=6)
        assert_parity(batch["obj"], got, ref, TOL[prec])
    # 0.x <= -1 excludes everything: every seventh LP is infeasible
    assert (ref["status"][::7] == oracle.INFEASIBLE).all()


@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP64])
@pytest.mark.parametrize("d", [3, 4, 5])
def test_lps_beyond_the_warp_stage(d, prec):
    # LPs above half of a CTA's stage run in the one-warp large-LP kernel, mixed with
    # small ones, 25 % infeasible; FP64 also follows the oracle's exact path
    half = lp2d.warp_stage_constraints_nd(d)
    sizes = np.array([half + 1, 2000, 5000, 40, 300, half + 1, 2000, 5000, 7, 3000] * 2)
    batch = workloads.ball_batch(d, sizes, seed=20 + d, infeasible_frac=0.25)
    want = prec == lp2d.PREC_FP64
    got = gpu_solve_nd(batch, seed=2, precision=prec, want=want)
    ref = oracle_nd(batch, seed=2, want_nviol=want)
    assert got["err"] == 0
    assert_parity(batch["obj"], got, ref, TOL[prec])
    if want:
        assert (got["nviol"] == ref["nviol"]).all()


@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP64])
def test_hand_solved_degenerate_golden(prec):
    # LPs whose optimum is not a point: the point returned is decided by the pivot's and
    # the start's tie rules (R23, R24) and the endpoint rule, and must be the
    # hand-derived one, in both visit orders where the case names one
    import lp_pins

    for case in lp_pins.load_hand_lps_nd():
        if case["solver"] != "nd":
            continue
        seed = 0 if case["order"] is None else lp_pins.seed_for_order(oracle.perm_array, case["order"])
        d = len(case["obj"])
        cons = np.asarray(case["cons"], np.float32)
        batch = {"a": np.ascontiguousarray(cons[:, :d].T), "b": cons[:, d].copy(),
                 "offsets": np.array([0, len(cons)], np.int64), "obj": np.asarray([case["obj"]], np.float32),
                 "box": case["box"]}
        got = gpu_solve_nd(batch, seed=seed, precision=prec)
        assert got["status"][0] == case["status"], case["name"]
        tol = 1e-12 if prec == lp2d.PREC_FP64 else 1e-6
        assert np.allclose(got["x"][0], case["x"], rtol=0, atol=tol), (case["name"], got["x"][0])
