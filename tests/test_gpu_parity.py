"""GPU parity: the CUDA solver (through the C ABI) against the FP64 CPU oracle on the
same seeded inputs.  Status is compared bit-exactly; the objective c.x within 1e-4
relative (FP32) or 1e-10 (FP64), relative to max(|f_oracle|, 1)."""
from __future__ import annotations

import os

import numpy as np
import pytest

import lp_pins

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1902_04995_gb300 import lp2d, workloads  # noqa: E402

TOL = {lp2d.PREC_FP32: 1e-4, lp2d.PREC_FP64: 1e-10}
THREADS = os.cpu_count() or 1
DEV = torch.device("cuda:0")


def to_dev(batch):
    return {k: torch.from_numpy(np.ascontiguousarray(batch[k])).to(DEV)
            for k in ("ax", "ay", "b", "offsets", "obj")}


def gpu_solve(batch, seed=0, precision=lp2d.PREC_FP32, schedule=lp2d.SCHED_PERSISTENT, want=False, **tune):
    t = to_dev(batch)
    n_lp = len(batch["offsets"]) - 1
    nviol = torch.full((max(n_lp, 1),), -7, dtype=torch.int32, device=DEV) if want else None
    dfn = torch.full((max(2 * n_lp, 1),), -7, dtype=torch.int32, device=DEV) if want else None
    opts = lp2d.default_options(seed=seed, precision=precision, schedule=schedule,
                                out_nviol=nviol.data_ptr() if want else None,
                                out_def=dfn.data_ptr() if want else None, **tune)
    out_dtype = torch.float64 if precision == lp2d.PREC_FP64 else torch.float32
    xy = torch.full((max(2 * n_lp, 1),), 12345.0, dtype=out_dtype, device=DEV)
    st = torch.full((max(n_lp, 1),), -9, dtype=torch.int32, device=DEV)
    ws = lp2d.new_workspace(n_lp, opts, device=DEV)
    lp2d.solve_batch_ex(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"], xy, st,
                        opts, ws)
    torch.cuda.synchronize()
    assert lp2d.read_device_error(ws) == 0
    res = {"xy": xy[:2 * n_lp].cpu().numpy().reshape(-1, 2).astype(np.float64), "status": st[:n_lp].cpu().numpy()}
    if want:
        res["nviol"] = nviol[:n_lp].cpu().numpy()
        res["def"] = dfn[:2 * n_lp].cpu().numpy().reshape(-1, 2)
    return res


def oracle_solve(batch, seed=0, **kw):
    return oracle.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"], batch["box"],
                              seed=seed, threads=THREADS, **kw)


def assert_parity(batch, got, ref, tol):
    st, rst = got["status"], ref["status"]
    bad = np.nonzero(st != rst)[0]
    assert bad.size == 0, f"{bad.size} status mismatches, first LPs {bad[:10]}: gpu {st[bad[:10]]} oracle {rst[bad[:10]]}"
    c = np.asarray(batch["obj"], np.float64).reshape(-1, 2)
    solved = (rst == oracle.OPTIMAL) | (rst == oracle.BOX_BOUNDED)
    f_ref = np.einsum("ij,ij->i", ref["xy"], c)[solved]
    f_got = np.einsum("ij,ij->i", got["xy"], c)[solved]
    err = np.abs(f_got - f_ref) / np.maximum(np.abs(f_ref), 1.0)
    assert err.size == 0 or err.max() <= tol, f"max rel objective error {err.max():.3e} > {tol}"
    # the returned vertex itself (unique for these generic inputs)
    scale = np.maximum(np.abs(ref["xy"][solved]).max(axis=1, initial=0), 1.0)
    verr = np.abs(got["xy"][solved] - ref["xy"][solved]).max(axis=1, initial=0) / scale
    assert verr.size == 0 or verr.max() <= 50 * tol, f"max rel vertex error {verr.max():.3e}"
    unsolved = ~solved
    assert np.isnan(got["xy"][unsolved]).all()
    return err.max(initial=0.0)


# --------------------------------------------------------------- visit order
@pytest.mark.parametrize("m", [1, 2, 3, 5, 17, 64, 255, 256, 257, 1000, 2048, 4097, 70000])
def test_visit_order_matches_oracle(m):
    out = torch.empty(m, dtype=torch.int64, device=DEV)
    for seed in (0, 5, 2**64 - 3, 20190213 + m):
        lp2d.visit_order(seed, m, out)
        torch.cuda.synchronize()
        assert (out.cpu().numpy() == oracle.perm_array(seed, m)).all()


# ------------------------------------------------------------ hand-solved LPs
@pytest.mark.parametrize("prec,sched", [(lp2d.PREC_FP32, lp2d.SCHED_PERSISTENT), (lp2d.PREC_FP32, lp2d.SCHED_UNIFORM),
                                        (lp2d.PREC_FP32_F64ISECT, lp2d.SCHED_PERSISTENT),
                                        (lp2d.PREC_FP64, lp2d.SCHED_PERSISTENT), (lp2d.PREC_FP64, lp2d.SCHED_UNIFORM)])
def test_hand_solved_golden(prec, sched):
    # seeds 0 and 2 visit the two constraints of the two-constraint LPs (among them the
    # pins of readings R2 and R3) in both orders
    for seed in (0, 2):
        for case in lp_pins.load_hand_lps():
            cons = np.asarray(case["cons"], np.float32).reshape(-1, 3)
            batch = {"ax": cons[:, 0].copy(), "ay": cons[:, 1].copy(), "b": cons[:, 2].copy(),
                     "offsets": np.array([0, len(cons)], np.int64), "obj": np.asarray([case["obj"]], np.float32),
                     "box": case["box"]}
            got = gpu_solve(batch, seed=seed, precision=prec, schedule=sched)
            assert got["status"][0] == case["status"], (case["name"], seed)
            if case["xyf"] is not None:
                x, y, f = case["xyf"]
                tol = 1e-12 if prec == lp2d.PREC_FP64 else 1e-5
                assert abs(got["xy"][0, 0] - x) <= tol * max(1, abs(x)), (case["name"], seed)
                assert abs(got["xy"][0, 1] - y) <= tol * max(1, abs(y)), (case["name"], seed)


# ------------------------------------------------------------ the workloads
@pytest.mark.parametrize("prec,sched", [(lp2d.PREC_FP32, lp2d.SCHED_PERSISTENT), (lp2d.PREC_FP32, lp2d.SCHED_UNIFORM),
                                        (lp2d.PREC_FP64, lp2d.SCHED_PERSISTENT), (lp2d.PREC_FP64, lp2d.SCHED_UNIFORM)])
def test_plain_small_256x64(prec, sched):
    batch = workloads.plain_small()
    got = gpu_solve(batch, seed=11, precision=prec, schedule=sched)
    ref = oracle_solve(batch, seed=11)
    assert_parity(batch, got, ref, TOL[prec])


@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP64])
def test_plain_65536x256_full(prec):
    batch = workloads.plain_at_scale()
    got = gpu_solve(batch, seed=0, precision=prec)
    ref = oracle_solve(batch, seed=0)
    assert (ref["status"] == oracle.INFEASIBLE).sum() == 6554
    assert_parity(batch, got, ref, TOL[prec])


def test_ragged_131072_full_fp32():
    batch = workloads.ragged()
    got = gpu_solve(batch, seed=0)
    ref = oracle_solve(batch, seed=0)
    assert_parity(batch, got, ref, TOL[lp2d.PREC_FP32])


def test_ragged_fp64_uniform_slice():
    batch = workloads.ragged(n_lp=8192)
    got = gpu_solve(batch, seed=3, precision=lp2d.PREC_FP64, schedule=lp2d.SCHED_UNIFORM)
    ref = oracle_solve(batch, seed=3)
    assert_parity(batch, got, ref, TOL[lp2d.PREC_FP64])


# ----------------------------------------------------------- control flow
@pytest.mark.parametrize("sched", [lp2d.SCHED_PERSISTENT, lp2d.SCHED_UNIFORM])
def test_fp64_violation_counts_and_defining_pair_match_oracle(sched):
    # Same pi, same FP64 arithmetic: the GPU takes the oracle's exact path.
    batch = workloads.ragged(n_lp=4096, lo=8, hi=3000)
    got = gpu_solve(batch, seed=5, precision=lp2d.PREC_FP64, schedule=sched, want=True)
    ref = oracle_solve(batch, seed=5, want_nviol=True, want_def=True)
    assert_parity(batch, got, ref, TOL[lp2d.PREC_FP64])
    assert (got["nviol"] == ref["nviol"]).all()
    solved = ref["status"] != oracle.INFEASIBLE
    assert (np.sort(got["def"][solved], 1) == np.sort(ref["def"][solved][:, :2], 1)).all()


def test_fp32_defining_pair_matches_oracle():
    # FP32 may pick another constraint through a (nearly) degenerate vertex, where two
    # constraints give sigma values within FP32 rounding; the objective still agrees.
    batch = workloads.plain_at_scale(n_lp=8192)
    got = gpu_solve(batch, seed=1, want=True)
    ref = oracle_solve(batch, seed=1, want_def=True, want_nviol=True)
    assert_parity(batch, got, ref, TOL[lp2d.PREC_FP32])
    solved = ref["status"] != oracle.INFEASIBLE
    same = (np.sort(got["def"][solved], 1) == np.sort(ref["def"][solved][:, :2], 1)).all(1)
    assert same.mean() >= 0.999
    assert abs(got["nviol"].mean() - ref["nviol"].mean()) < 0.05 * ref["nviol"].mean()


@pytest.mark.parametrize("prec,sched", [(lp2d.PREC_FP32, lp2d.SCHED_PERSISTENT),
                                        (lp2d.PREC_FP32_F64ISECT, lp2d.SCHED_PERSISTENT),
                                        (lp2d.PREC_FP64, lp2d.SCHED_PERSISTENT), (lp2d.PREC_FP64, lp2d.SCHED_UNIFORM)])
def test_ties_go_to_the_earliest_position(prec, sched):
    # Reading R3 through out_def: every LP carries an exact copy of a constraint through
    # its optimum; equal sigma values of the two copies must resolve to the copy the
    # oracle reports (the earlier-visited one), on every LP whose defining pair holds
    # one of them.
    import test_oracle_pins

    batch, pair = test_oracle_pins.duplicate_defining_constraint_batch(oracle, 3000, seed=41)
    got = gpu_solve(batch, seed=6, precision=prec, schedule=sched, want=True)
    ref = oracle_solve(batch, seed=6, want_def=True)
    assert_parity(batch, got, ref, TOL[lp2d.PREC_FP64] if prec == lp2d.PREC_FP64 else TOL[lp2d.PREC_FP32])
    solved = ref["status"] != oracle.INFEASIBLE
    rdef = np.sort(ref["def"][:, :2], 1)
    gdef = np.sort(got["def"], 1)
    involved = solved & ((rdef == pair[:, :1]) | (rdef == pair[:, 1:])).any(1)
    assert involved.sum() >= 2000
    bad = np.nonzero(involved & (rdef != gdef).any(1))[0]
    assert bad.size == 0, (bad[:8], rdef[bad[:8]], gdef[bad[:8]], pair[bad[:8]])


def test_results_identical_across_tuning():
    batch = workloads.ragged(n_lp=20000)
    base = gpu_solve(batch, seed=2)
    for tune in ({"ctas_per_sm": 1}, {"ctas_per_sm": 3, "chunk_big": 1, "chunk_small": 1},
                 {"chunk_big": 16, "chunk_small": 8}, {"team_min_slots": 64}, {"team_min_slots": 4096},
                 {"l2_prefetch": -1, "team_min_slots": 300}, {"lane_max_m": -1}, {"lane_max_m": 1},
                 {"lane_max_m": 16, "chunk_small": 1}):
        got = gpu_solve(batch, seed=2, **tune)
        assert (got["status"] == base["status"]).all()
        assert np.array_equal(got["xy"], base["xy"], equal_nan=True), tune


@pytest.mark.parametrize("lo,hi,n_lp", [(8, 16, 20000), (513, 1024, 3000), (1025, 2060, 2000), (1, 8, 30000)])
def test_batches_of_one_size_class(lo, hi, n_lp):
    # every LP in one size class: the queue of that class is dense and the others are
    # empty, so each phase's grab spans take their extreme values
    rng = np.random.default_rng(lo * 7 + hi)
    sizes = rng.integers(lo, hi + 1, n_lp)
    batch = workloads.disk_batch(sizes, seed=lo + hi, infeasible_frac=0.1)
    base = gpu_solve(batch, seed=4)
    assert_parity(batch, base, oracle_solve(batch, seed=4), TOL[lp2d.PREC_FP32])
    for tune in ({"chunk_big": 32, "chunk_small": 16}, {"chunk_big": 1, "chunk_small": 1, "ctas_per_sm": 2},
                 {"lane_max_m": -1}, {"lane_max_m": 16}):
        got = gpu_solve(batch, seed=4, **tune)
        assert (got["status"] == base["status"]).all(), tune
        assert np.array_equal(got["xy"], base["xy"], equal_nan=True), tune


@pytest.mark.parametrize("lane_max_m", [8, 16])
def test_single_lane_lps_match_whole_warps(lane_max_m):
    # LPs of 0..16 constraints (a tenth infeasible, a few with NaN data) among larger
    # ones, solved one per lane and one per warp: the same statuses, vertices, violation
    # counts and defining constraints, bit for bit, and the oracle's results.
    rng = np.random.default_rng(lane_max_m)
    sizes = np.concatenate([np.arange(0, 17), rng.integers(0, lane_max_m + 1, 20000), rng.integers(1, 200, 3000)])
    rng.shuffle(sizes)
    batch = workloads.disk_batch(sizes, seed=77, infeasible_frac=0.1)
    starts = batch["offsets"][:-1][sizes > 3]
    batch["ax"][starts[::501] + 1] = np.nan
    lanes = gpu_solve(batch, seed=8, want=True, lane_max_m=lane_max_m)
    whole = gpu_solve(batch, seed=8, want=True, lane_max_m=-1)
    assert (lanes["status"] == whole["status"]).all()
    assert np.array_equal(lanes["xy"], whole["xy"], equal_nan=True)
    assert (lanes["nviol"] == whole["nviol"]).all()
    ok = (whole["status"] == oracle.OPTIMAL) | (whole["status"] == oracle.BOX_BOUNDED)
    assert (lanes["def"][ok] == whole["def"][ok]).all()
    ref = oracle_solve(batch, seed=8, want_def=True)
    assert (ref["status"] == oracle.BAD_INPUT).sum() == starts[::501].size
    assert_parity(batch, lanes, ref, TOL[lp2d.PREC_FP32])
    solved = ref["status"] != oracle.INFEASIBLE
    same = (np.sort(lanes["def"][solved & ok], 1) == np.sort(ref["def"][solved & ok][:, :2], 1)).all(1)
    assert same.mean() >= 0.999


def test_autotune_picks_a_grid_point_and_keeps_the_results():
    batch = workloads.ragged(n_lp=20000)
    t = to_dev(batch)
    base = gpu_solve(batch, seed=2)
    solver = lp2d.Solver(20000, lp2d.default_options(seed=2), device=DEV)
    ms = solver.autotune(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"], reps=2)
    o = solver.options
    assert ms > 0.0
    assert o.chunk_big in (1, 2, 4) and o.chunk_small in (1, 2, 4, 8) and o.ctas_per_sm >= 1
    assert o.team_min_slots in (512, 1024, 4096)
    assert o.lane_max_m in (-1, 8, 16)
    solver(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"])
    torch.cuda.synchronize()
    assert (solver.out_status.cpu().numpy() == base["status"]).all()
    assert np.array_equal(solver.out_xy.cpu().numpy().reshape(-1, 2).astype(np.float64), base["xy"], equal_nan=True)
    with pytest.raises(lp2d.LP2DError):
        lp2d.autotune(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"], solver.out_xy,
                      solver.out_status, lp2d.default_options(schedule=lp2d.SCHED_UNIFORM), solver.workspace)


def test_repeated_launches_reuse_workspace_and_graph_replay_is_identical():
    batch = workloads.ragged(n_lp=30000)
    t = to_dev(batch)
    n_lp = len(batch["offsets"]) - 1
    solver = lp2d.Solver(n_lp, lp2d.default_options(seed=9), device=DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(3):
            solver(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"])
    s.synchronize()
    eager = (solver.out_xy.clone(), solver.out_status.clone())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        solver(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"])
    solver.out_xy.zero_()
    solver.out_status.zero_()
    for _ in range(5):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(solver.out_status, eager[1])
    assert torch.equal(torch.nan_to_num(solver.out_xy, nan=7.0), torch.nan_to_num(eager[0], nan=7.0))
    ref = oracle_solve(batch, seed=9)
    got = {"xy": solver.out_xy.cpu().numpy().reshape(-1, 2).astype(np.float64), "status": solver.out_status.cpu().numpy()}
    assert_parity(batch, got, ref, TOL[lp2d.PREC_FP32])
    assert lp2d.read_device_error(solver.workspace) == 0


# ----------------------------------------------------------- edge cases
def test_ragged_edges_tiles_and_tails():
    # sizes straddling the warp (32), team (128), quarter-stage (512), half-stage (1024)
    # and CTA-stage (2060) boundaries, plus LPs beyond the stage that read through pi
    # from HBM.
    sizes = np.array([0, 1, 2, 3, 4, 31, 32, 33, 63, 64, 65, 127, 128, 129, 511, 512, 513, 1023, 1024, 1025,
                      2047, 2048, 2049, 2059, 2060, 2061, 3000, 9000], dtype=np.int64)
    sizes = np.concatenate([sizes, sizes[::-1], sizes])
    batch = workloads.disk_batch(sizes, seed=4, infeasible_frac=0.3)
    for prec in (lp2d.PREC_FP32, lp2d.PREC_FP64):
        for sched in (lp2d.SCHED_PERSISTENT, lp2d.SCHED_UNIFORM):
            got = gpu_solve(batch, seed=1, precision=prec, schedule=sched)
            ref = oracle_solve(batch, seed=1)
            assert_parity(batch, got, ref, TOL[prec])


def test_single_huge_lp_reads_through_global_memory():
    batch = workloads.disk_batch(np.array([60000], np.int64), seed=8, infeasible_frac=1.0)
    got = gpu_solve(batch, seed=1)
    ref = oracle_solve(batch, seed=1)
    assert ref["status"][0] == oracle.INFEASIBLE
    assert_parity(batch, got, ref, TOL[lp2d.PREC_FP32])
    batch = workloads.disk_batch(np.array([60000, 5], np.int64), seed=9)
    assert_parity(batch, gpu_solve(batch, seed=2), oracle_solve(batch, seed=2), TOL[lp2d.PREC_FP32])


def test_empty_batch_is_noop():
    batch = workloads.disk_batch(np.zeros(0, np.int64), seed=1)
    got = gpu_solve(batch)
    assert got["status"].size == 0


def test_bad_input_and_bad_offsets():
    batch = workloads.disk_batch(np.array([10, 10, 10, 600, 10], np.int64), seed=3)
    batch["ax"][3] = np.nan          # LP 0
    batch["b"][25] = np.inf          # LP 2
    batch["ay"][40] = -np.inf        # LP 3 (team path)
    got = gpu_solve(batch)
    ref = oracle_solve(batch)
    assert list(ref["status"][[0, 2, 3]]) == [oracle.BAD_INPUT] * 3
    assert (got["status"] == ref["status"]).all()
    assert np.isnan(got["xy"][[0, 2, 3]]).all()
    # a decreasing offset gives that LP BAD_INPUT and sets the device error bit
    bad = dict(batch)
    bad["ax"] = np.nan_to_num(batch["ax"]).astype(np.float32)
    bad["ay"] = np.nan_to_num(batch["ay"]).astype(np.float32)
    bad["b"] = np.nan_to_num(batch["b"], posinf=1.0).astype(np.float32)
    off = bad["offsets"].copy()
    off[2] = off[1] - 3
    bad["offsets"] = off
    t = to_dev(bad)
    n_lp = 5
    xy = torch.empty(10, dtype=torch.float32, device=DEV)
    st = torch.empty(5, dtype=torch.int32, device=DEV)
    ws = lp2d.new_workspace(n_lp, device=DEV)
    lp2d.solve_batch_ex(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), bad["box"], xy, st, None, ws)
    assert lp2d.read_device_error(ws) & lp2d.DEVERR_BAD_OFFSETS
    assert st[1].item() == lp2d.BAD_INPUT
    assert lp2d.read_device_error(ws) == 0  # reading clears it


@pytest.mark.parametrize("lane_max_m", [-1, 16])
def test_non_finite_objective_and_empty_lps_in_every_class(lane_max_m):
    # a NaN or infinite objective gives BAD_INPUT whatever the LP's size class (one
    # thread, one warp, half a CTA, a CTA); empty LPs end at the box corner
    sizes = np.array([0, 1, 5, 16, 17, 40, 512, 700, 1500, 2049, 0, 5, 40, 700, 1500], np.int64)
    batch = workloads.disk_batch(sizes, seed=12)
    batch["obj"] = batch["obj"].copy()
    batch["obj"][[2, 5, 7, 8]] = [[np.nan, 1.0], [1.0, np.inf], [-np.inf, 0.0], [np.nan, np.nan]]
    got = gpu_solve(batch, seed=3, lane_max_m=lane_max_m)
    ref = oracle_solve(batch, seed=3)
    assert list(ref["status"][[2, 5, 7, 8]]) == [oracle.BAD_INPUT] * 4
    assert (got["status"] == ref["status"]).all()
    assert np.isnan(got["xy"][[2, 5, 7, 8]]).all()
    assert list(ref["status"][[0, 10]]) == [oracle.BOX_BOUNDED] * 2
    ok = ref["status"] != oracle.BAD_INPUT
    c = np.asarray(batch["obj"], np.float64)[ok]
    f_got = np.einsum("ij,ij->i", got["xy"][ok], c)
    f_ref = np.einsum("ij,ij->i", ref["xy"][ok], c)
    solved = (ref["status"][ok] == oracle.OPTIMAL) | (ref["status"][ok] == oracle.BOX_BOUNDED)
    assert (np.abs(f_got - f_ref)[solved] <= TOL[lp2d.PREC_FP32] * np.maximum(np.abs(f_ref[solved]), 1.0)).all()


def test_short_form_entry_point():
    batch = workloads.plain_small(seed=77)
    t = to_dev(batch)
    n_lp = len(batch["offsets"]) - 1
    xy = torch.empty(2 * n_lp, dtype=torch.float32, device=DEV)
    st = torch.empty(n_lp, dtype=torch.int32, device=DEV)
    for _ in range(2):
        lp2d.solve_batch(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"].reshape(-1), batch["box"], xy, st)
    torch.cuda.synchronize()
    got = {"xy": xy.cpu().numpy().reshape(-1, 2).astype(np.float64), "status": st.cpu().numpy()}
    assert_parity(batch, got, oracle_solve(batch, seed=0), TOL[lp2d.PREC_FP32])


# ------------------------------------------------- precision (near-parallel)
@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP32_F64ISECT, lp2d.PREC_FP64])
def test_collision_workload_every_mode(prec):
    # 16-gon speed limits plus neighbour half-planes, 5 % of them within 1e-6 rad of
    # an earlier normal: every precision mode matches the oracle (status exact,
    # objective within 1e-4 for the FP32 modes and 1e-10 for FP64).
    batch = workloads.collision()
    got = gpu_solve(batch, seed=4, precision=prec)
    ref = oracle_solve(batch, seed=4)
    assert_parity(batch, got, ref, TOL[lp2d.PREC_FP64] if prec == lp2d.PREC_FP64 else TOL[lp2d.PREC_FP32])


def test_mixed_precision_on_plain_and_ragged():
    for batch in (workloads.plain_at_scale(n_lp=8192), workloads.ragged(n_lp=8192, hi=3000)):
        got = gpu_solve(batch, seed=6, precision=lp2d.PREC_FP32_F64ISECT)
        assert_parity(batch, got, oracle_solve(batch, seed=6), TOL[lp2d.PREC_FP32])


def test_near_parallel_pair_mixed_mode():
    # Two constraints whose normals differ by about 1e-7 rad cross far away; the FP32
    # determinant of such a pair is pure rounding, the mixed mode recomputes it.
    rng = np.random.default_rng(12)
    n = 512
    ang = rng.uniform(0, 2 * np.pi, n)
    d = np.float32(1e-7)
    cons = []
    for a in ang:
        n1 = np.array([np.cos(a), np.sin(a)], np.float32)
        n2 = np.array([np.cos(a + d), np.sin(a + d)], np.float32)
        cons += [[n1[0], n1[1], 1.0], [n2[0], n2[1], 1.0], [-n1[0], -n1[1], 3.0]]
    cons = np.asarray(cons, np.float32)
    batch = {"ax": cons[:, 0].copy(), "ay": cons[:, 1].copy(), "b": cons[:, 2].copy(),
             "offsets": np.arange(0, 3 * n + 1, 3, dtype=np.int64),
             "obj": np.stack([np.cos(ang + 1.5), np.sin(ang + 1.5)], 1).astype(np.float32), "box": (-1e3, 1e3, -1e3, 1e3)}
    ref = oracle_solve(batch, seed=2)
    got = gpu_solve(batch, seed=2, precision=lp2d.PREC_FP32_F64ISECT)
    assert (got["status"] == ref["status"]).all()
    # plain FP32 on the same LPs: these optima lie on a box side, where the pair's
    # rounding does not reach the status, so FP32 agrees here as well
    got32 = gpu_solve(batch, seed=2, precision=lp2d.PREC_FP32)
    assert (got32["status"] == ref["status"]).all()


def _mismatches(batch, got, ref, tol):
    """(status mismatches, LPs whose objective misses the tolerance)."""
    st = int((got["status"] != ref["status"]).sum())
    c = np.asarray(batch["obj"], np.float64).reshape(-1, 2)
    ok = (ref["status"] != oracle.INFEASIBLE) & (got["status"] != oracle.INFEASIBLE)
    f_ref = np.einsum("ij,ij->i", ref["xy"][ok], c[ok])
    f_got = np.einsum("ij,ij->i", got["xy"][ok], c[ok])
    return st, int((np.abs(f_got - f_ref) / np.maximum(np.abs(f_ref), 1.0) > tol).sum())


def test_mixed_mode_resolves_what_fp32_cannot():
    # The optimum of every LP is the crossing of two lines about 1e-5 rad apart, 0.1 %
    # inside or outside the box (workloads.near_parallel_pairs): FP32 places the
    # crossing only to about 2^-24 / 1e-5 = 0.6 %, so it misjudges feasibility and the
    # objective; FP32 with FP64 intersections and FP64 match the oracle on every LP.
    batch = workloads.near_parallel_pairs(4096, seed=3)
    ref = oracle_solve(batch, seed=3)
    assert (ref["status"] == oracle.INFEASIBLE).sum() == 2048
    mixed = gpu_solve(batch, seed=3, precision=lp2d.PREC_FP32_F64ISECT)
    assert_parity(batch, mixed, ref, TOL[lp2d.PREC_FP32])
    assert_parity(batch, gpu_solve(batch, seed=3, precision=lp2d.PREC_FP64), ref, TOL[lp2d.PREC_FP64])
    st32, f32 = _mismatches(batch, gpu_solve(batch, seed=3, precision=lp2d.PREC_FP32), ref, TOL[lp2d.PREC_FP32])
    print(f"plain FP32 on near-parallel pairs: {st32} status mismatches, {f32} objectives beyond 1e-4")
    assert st32 + f32 >= 100


def test_mixed_precision_needs_persistent_schedule():
    batch = workloads.plain_small()
    with pytest.raises(lp2d.LP2DError) as e:
        gpu_solve(batch, precision=lp2d.PREC_FP32_F64ISECT, schedule=lp2d.SCHED_UNIFORM)
    assert e.value.code == lp2d.ERR_UNSUPPORTED


# --------------------------------------------------------- degenerate inputs
@pytest.mark.parametrize("prec,sched", [(lp2d.PREC_FP32, lp2d.SCHED_PERSISTENT), (lp2d.PREC_FP64, lp2d.SCHED_PERSISTENT),
                                        (lp2d.PREC_FP32_F64ISECT, lp2d.SCHED_PERSISTENT),
                                        (lp2d.PREC_FP64, lp2d.SCHED_UNIFORM)])
def test_degenerate_lifted_duplicate_and_zero_normal_constraints(prec, sched):
    """1-D LPs lifted to 2-D (a_y = 0, c_y = 0: segment optima, BOX_BOUNDED), then LPs
    with exact duplicate and zero-normal constraints; status exact, objective within
    the mode's tolerance (the vertex of a segment optimum is not unique)."""
    rng = np.random.default_rng(71)
    tol = 1e-10 if prec == lp2d.PREC_FP64 else 1e-4

    def check(batch, seed):
        got = gpu_solve(batch, seed=seed, precision=prec, schedule=sched)
        ref = oracle_solve(batch, seed=seed)
        assert np.array_equal(got["status"], ref["status"]), np.nonzero(got["status"] != ref["status"])[0][:8]
        c = np.asarray(batch["obj"], np.float64).reshape(-1, 2)
        ok = ref["status"] != oracle.INFEASIBLE
        f_ref = np.einsum("ij,ij->i", ref["xy"][ok], c[ok])
        f_got = np.einsum("ij,ij->i", got["xy"][ok], c[ok])
        assert (np.abs(f_got - f_ref) / np.maximum(np.abs(f_ref), 1.0)).max(initial=0.0) <= tol
        assert np.isnan(got["xy"][~ok]).all()
        return ref

    sizes = workloads.loguniform_sizes(rng, 800, 1, 1500)
    offsets = np.zeros(801, np.int64)
    np.cumsum(sizes, out=offsets[1:])
    n = int(offsets[-1])
    sgn = np.where(rng.random(n) < 0.5, -1.0, 1.0).astype(np.float32)
    lifted = {"ax": sgn, "ay": np.zeros(n, np.float32), "b": rng.uniform(0.5, 3.0, n).astype(np.float32),
              "offsets": offsets,
              "obj": np.stack([np.where(rng.random(800) < 0.5, -1.0, 1.0), np.zeros(800)], 1).astype(np.float32),
              "box": (-1e3, 1e3, -7.0, 3.0)}
    ref = check(lifted, 2)
    assert (ref["status"] == oracle.BOX_BOUNDED).all()
    base = workloads.disk_batch(np.full(300, 60), seed=72, infeasible_frac=0.1)
    cols = {k: [] for k in ("ax", "ay", "b")}
    sz = []
    for l in range(300):
        s, e = base["offsets"][l], base["offsets"][l + 1]
        dup = rng.choice(e - s, size=10)
        extra_b = np.array([1.0, 1.0, -1.0 if l % 7 == 0 else 2.0], np.float32)
        perm = rng.permutation(e - s + 13)
        for k in ("ax", "ay"):
            v = base[k][s:e]
            cols[k].append(np.r_[v, v[dup], np.zeros(3, np.float32)][perm])
        cols["b"].append(np.r_[base["b"][s:e], base["b"][s:e][dup], extra_b][perm].astype(np.float32))
        sz.append(e - s + 13)
    off2 = np.zeros(301, np.int64)
    np.cumsum(sz, out=off2[1:])
    batch = {k: np.concatenate(v).astype(np.float32) for k, v in cols.items()}
    batch.update({"offsets": off2, "obj": base["obj"], "box": base["box"]})
    ref = check(batch, 3)
    assert (ref["status"][::7] == oracle.INFEASIBLE).all()
