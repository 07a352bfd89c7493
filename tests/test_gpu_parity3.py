"""GPU parity of the batched 3-D solver (lp3d_solve_batch_ex) against the FP64 3-D
oracle on the same seeded inputs: status bit-exact, the objective within 1e-4
relative (FP32) or 1e-10 (FP64) of max(|f_oracle|, 1); in FP64 also the number of
violations and the three defining constraints."""
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
TOL = {lp2d.PREC_FP32: 1e-4, lp2d.PREC_FP64: 1e-10}


def gpu_solve3(batch, seed=0, precision=lp2d.PREC_FP32, want=False, **tune):
    t = {k: torch.from_numpy(np.ascontiguousarray(batch[k]).reshape(-1)).to(DEV)
         for k in ("ax", "ay", "az", "b", "offsets", "obj")}
    n_lp = len(batch["offsets"]) - 1
    nviol = torch.full((max(n_lp, 1),), -7, dtype=torch.int32, device=DEV) if want else None
    dfn = torch.full((max(3 * n_lp, 1),), -7, dtype=torch.int32, device=DEV) if want else None
    opts = lp2d.default_options(seed=seed, precision=precision, out_nviol=nviol.data_ptr() if want else None,
                                out_def=dfn.data_ptr() if want else None, **tune)
    dt = torch.float64 if precision == lp2d.PREC_FP64 else torch.float32
    xyz = torch.full((max(3 * n_lp, 1),), 12345.0, dtype=dt, device=DEV)
    st = torch.full((max(n_lp, 1),), -9, dtype=torch.int32, device=DEV)
    ws = lp2d.new_workspace(n_lp, opts, device=DEV)
    lp2d.solve_batch3d(t["ax"], t["ay"], t["az"], t["b"], t["offsets"], t["obj"], batch["box"], xyz, st, opts, ws)
    torch.cuda.synchronize()
    res = {"xyz": xyz[:3 * n_lp].cpu().numpy().reshape(-1, 3).astype(np.float64), "status": st[:n_lp].cpu().numpy(),
           "err": lp2d.read_device_error(ws)}
    if want:
        res["nviol"] = nviol[:n_lp].cpu().numpy()
        res["def"] = dfn[:3 * n_lp].cpu().numpy().reshape(-1, 3)
    return res


def oracle3(batch, seed=0, **kw):
    return oracle.solve_batch3(batch["ax"], batch["ay"], batch["az"], batch["b"], batch["offsets"], batch["obj"],
                               batch["box"], seed=seed, threads=THREADS, **kw)


def assert_parity3(batch, got, ref, tol):
    bad = np.nonzero(got["status"] != ref["status"])[0]
    assert bad.size == 0, f"{bad.size} status mismatches, first {bad[:8]}: gpu {got['status'][bad[:8]]} oracle {ref['status'][bad[:8]]}"
    c = batch["obj"].astype(np.float64)
    solved = (ref["status"] == oracle.OPTIMAL) | (ref["status"] == oracle.BOX_BOUNDED)
    f_ref = np.einsum("ij,ij->i", ref["xyz"], c)[solved]
    f_got = np.einsum("ij,ij->i", got["xyz"], c)[solved]
    err = np.abs(f_got - f_ref) / np.maximum(np.abs(f_ref), 1.0)
    assert err.size == 0 or err.max() <= tol, f"max rel objective error {err.max():.3e}"
    assert np.isnan(got["xyz"][~solved]).all()
    return err.max(initial=0.0)


@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP64])
def test_small_batches_match_the_oracle(prec):
    for sizes, seed in ((np.full(512, 40), 1), (workloads.loguniform_sizes(np.random.default_rng(5), 3000, 1, 1018), 2)):
        batch = workloads.sphere_batch(sizes, seed=seed, infeasible_frac=0.1)
        assert_parity3(batch, gpu_solve3(batch, seed=3, precision=prec), oracle3(batch, seed=3), TOL[prec])


def test_fp64_violation_counts_and_defining_planes_match_the_oracle():
    batch = workloads.sphere_batch(workloads.loguniform_sizes(np.random.default_rng(6), 2000, 1, 1018), seed=4,
                                   infeasible_frac=0.1)
    got = gpu_solve3(batch, seed=5, precision=lp2d.PREC_FP64, want=True)
    ref = oracle3(batch, seed=5, want_def=True, want_nviol=True)
    assert_parity3(batch, got, ref, TOL[lp2d.PREC_FP64])
    # the same FP64 steps in the same order, ties included (R17, R18): the oracle's path
    assert (got["nviol"] == ref["nviol"]).all()
    ok = ref["status"] != oracle.INFEASIBLE
    assert (np.sort(got["def"][ok], 1) == np.sort(ref["def"][ok], 1)).all()


def test_plain3d_at_scale():
    batch = workloads.plain3d()
    got = gpu_solve3(batch, seed=0)
    assert_parity3(batch, got, oracle3(batch, seed=0), TOL[lp2d.PREC_FP32])
    assert got["err"] == 0


def test_ragged3d_at_scale():
    batch = workloads.ragged3d()
    got = gpu_solve3(batch, seed=0)
    assert_parity3(batch, got, oracle3(batch, seed=0), TOL[lp2d.PREC_FP32])


def test_edge_cases_empty_tiny_bad_and_too_large():
    # the class boundaries (quarter and half stage), the large-LP kernel (1019 and up)
    # and its cap (12282), and one LP above it
    sizes = np.array([0, 1, 2, 3, 6, 31, 32, 33, 505, 506, 507, 1018, 1019, 2000, 5000, 12282, 12283])
    batch = workloads.sphere_batch(sizes, seed=7)
    got = gpu_solve3(batch, seed=1)
    ref = oracle3(batch, seed=1)
    keep = sizes <= lp2d.MAX_CONSTRAINTS_3D
    assert (got["status"][~keep] == oracle.BAD_INPUT).all()
    assert got["err"] & lp2d.DEVERR_TOO_LARGE
    bad = np.nonzero(got["status"][keep] != ref["status"][keep])[0]
    assert bad.size == 0, bad
    c = batch["obj"].astype(np.float64)
    solved = keep & (ref["status"] != oracle.INFEASIBLE)
    f_ref = np.einsum("ij,ij->i", ref["xyz"][solved], c[solved])
    f_got = np.einsum("ij,ij->i", got["xyz"][solved], c[solved])
    assert (np.abs(f_got - f_ref) / np.maximum(np.abs(f_ref), 1)).max() <= 1e-4
    # NaN data and a reversed LP (negative size) are BAD_INPUT
    b2 = workloads.sphere_batch(np.array([10, 10, 10]), seed=8)
    b2["ax"][12] = np.nan
    got = gpu_solve3(b2)
    assert got["status"][1] == oracle.BAD_INPUT and got["status"][0] != oracle.BAD_INPUT
    b2["offsets"] = np.array([0, 10, 5, 30], np.int64)
    got = gpu_solve3(b2)
    assert got["status"][1] == oracle.BAD_INPUT and got["err"] & lp2d.DEVERR_BAD_OFFSETS


def test_results_identical_across_tuning_and_repeated_launches():
    batch = workloads.sphere_batch(workloads.loguniform_sizes(np.random.default_rng(3), 5000, 4, 1018), seed=9,
                                   infeasible_frac=0.1)
    base = gpu_solve3(batch, seed=2)
    for tune in ({"chunk_small": 1}, {"chunk_small": 16, "ctas_per_sm": 1}):
        got = gpu_solve3(batch, seed=2, **tune)
        assert (got["status"] == base["status"]).all()
        assert np.array_equal(got["xyz"], base["xyz"], equal_nan=True)
    # the workspace is reused without a memset
    t = {k: torch.from_numpy(np.ascontiguousarray(batch[k]).reshape(-1)).to(DEV)
         for k in ("ax", "ay", "az", "b", "offsets", "obj")}
    n = len(batch["offsets"]) - 1
    opts = lp2d.default_options(seed=2)
    ws = lp2d.new_workspace(n, opts, device=DEV)
    xyz = torch.empty(3 * n, device=DEV)
    st = torch.empty(n, dtype=torch.int32, device=DEV)
    for _ in range(3):
        lp2d.solve_batch3d(t["ax"], t["ay"], t["az"], t["b"], t["offsets"], t["obj"], batch["box"], xyz, st, opts, ws)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == base["status"]).all()


def test_least_violation_of_infeasible_2d_lps():
    import lp_pins

    batch = workloads.ragged(n_lp=20000, hi=1017, seed=31)
    t = {k: torch.from_numpy(np.ascontiguousarray(batch[k]).reshape(-1)).to(DEV) for k in ("ax", "ay", "b", "offsets", "obj")}
    n = len(batch["offsets"]) - 1
    opts = lp2d.default_options(seed=3)
    ws = lp2d.new_workspace(n, opts, device=DEV)
    xy = torch.empty(2 * n, device=DEV)
    st = torch.empty(n, dtype=torch.int32, device=DEV)
    lp2d.solve_batch_ex(t["ax"], t["ay"], t["b"], t["offsets"], t["obj"], batch["box"], xy, st, opts, ws)
    st_lv = torch.full((n,), -5, dtype=torch.int32, device=DEV)
    tt = torch.full((n,), -5.0, device=DEV)
    lp2d.least_violation(t["ax"], t["ay"], t["b"], t["offsets"], batch["box"], st, xy, st_lv, out_t=tt,
                         options=lp2d.default_options(seed=3), workspace=ws)
    torch.cuda.synchronize()
    st2 = st.cpu().numpy()
    inf = st2 == oracle.INFEASIBLE
    assert inf.sum() > 1500
    lv = lp_pins.least_violation_batch(batch)
    ref = oracle.solve_batch3(lv["ax"], lv["ay"], lv["az"], lv["b"], lv["offsets"], lv["obj"], lv["box"], seed=3,
                              threads=THREADS)
    got_st, got_t, got_xy = st_lv.cpu().numpy(), tt.cpu().numpy(), xy.cpu().numpy().reshape(-1, 2)
    assert (got_st[~inf] == -5).all() and (got_t[~inf] == -5.0).all()  # untouched
    assert np.array_equal(got_st[inf], ref["status"][inf])
    tref = ref["xyz"][inf, 2]
    assert np.abs(got_t[inf] - tref).max() / max(np.abs(tref).max(), 1.0) <= 1e-4
    # the returned point violates no constraint by more than its t
    off = batch["offsets"]
    for l in np.nonzero(inf)[0][:300]:
        s, e = off[l], off[l + 1]
        a = np.stack([batch["ax"][s:e], batch["ay"][s:e]], 1).astype(np.float64)
        viol = (a @ got_xy[l].astype(np.float64) - batch["b"][s:e]) / np.linalg.norm(a, axis=1)
        assert viol.max() <= got_t[l] + 1e-3 * max(1.0, abs(got_t[l]))


def test_least_violation_in_fp64():
    import lp_pins

    batch = workloads.disk_batch(np.full(3000, 80), seed=41, infeasible_frac=0.3)
    t = {k: torch.from_numpy(np.ascontiguousarray(batch[k]).reshape(-1)).to(DEV) for k in ("ax", "ay", "b", "offsets", "obj")}
    n = len(batch["offsets"]) - 1
    st = torch.from_numpy(np.where(batch["infeasible"], 1, 0).astype(np.int32)).to(DEV)
    xy = torch.full((2 * n,), 7.0, dtype=torch.float64, device=DEV)
    st_lv = torch.full((n,), -5, dtype=torch.int32, device=DEV)
    tt = torch.full((n,), -5.0, device=DEV)
    opts = lp2d.default_options(precision=lp2d.PREC_FP64, seed=4)
    lp2d.least_violation(t["ax"], t["ay"], t["b"], t["offsets"], batch["box"], st, xy, st_lv, out_t=tt,
                         options=opts, workspace=lp2d.new_workspace(n, opts, device=DEV))
    torch.cuda.synchronize()
    inf = batch["infeasible"]
    lv = lp_pins.least_violation_batch(batch)
    ref = oracle.solve_batch3(lv["ax"], lv["ay"], lv["az"], lv["b"], lv["offsets"], lv["obj"], lv["box"], seed=4,
                              threads=THREADS)
    got_st, got_xy = st_lv.cpu().numpy(), xy.cpu().numpy().reshape(-1, 2)
    assert np.array_equal(got_st[inf], ref["status"][inf])
    assert (got_st[~inf] == -5).all() and (got_xy[~inf] == 7.0).all()
    f_ref = ref["xyz"][inf, 2]
    # the FP64 run reproduces the oracle's least violation (t is returned in float32)
    assert np.abs(tt.cpu().numpy()[inf] - f_ref).max() <= 1e-6 * max(1.0, np.abs(f_ref).max())
    # the returned point violates no constraint by more than the least violation
    off = batch["offsets"]
    for l in np.nonzero(inf)[0][:200]:
        s0, e0 = off[l], off[l + 1]
        a = np.stack([batch["ax"][s0:e0], batch["ay"][s0:e0]], 1).astype(np.float64)
        # |a| as the least-violation LP defines it (float32)
        viol = (a @ got_xy[l] - batch["b"][s0:e0]) / -lv["az"][s0:e0].astype(np.float64)
        assert viol.max() <= ref["xyz"][l, 2] + 1e-9


@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP64])
def test_degenerate_lifted_and_duplicate_constraints(prec):
    # 2-D LPs lifted to 3-D (az = 0, c_z = 0): every optimum is a segment along z,
    # BOX_BOUNDED on both sides; then exact duplicates and zero-normal constraints
    rng = np.random.default_rng(61)
    low = workloads.disk_batch(workloads.loguniform_sizes(rng, 800, 1, 500), seed=62, infeasible_frac=0.15)
    n = low["ax"].shape[0]
    lifted = {"ax": low["ax"], "ay": low["ay"], "az": np.zeros(n, np.float32), "b": low["b"],
              "offsets": low["offsets"], "obj": np.hstack([low["obj"], np.zeros((800, 1), np.float32)]),
              "box": tuple(low["box"]) + (-7.0, 3.0)}
    got = gpu_solve3(lifted, seed=2, precision=prec)
    ref = oracle3(lifted, seed=2)
    assert_parity3(lifted, got, ref, TOL[prec])
    assert (got["status"][ref["status"] != oracle.INFEASIBLE] == oracle.BOX_BOUNDED).all()
    base = workloads.sphere_batch(np.full(300, 60), seed=63, infeasible_frac=0.1)
    cols = {k: [] for k in ("ax", "ay", "az", "b")}
    sizes = []
    for l in range(300):
        s, e = base["offsets"][l], base["offsets"][l + 1]
        dup = rng.choice(e - s, size=10)
        extra_b = np.array([1.0, 1.0, -1.0 if l % 7 == 0 else 2.0], np.float32)
        perm = rng.permutation(e - s + 13)
        for k in ("ax", "ay", "az"):
            v = base[k][s:e]
            cols[k].append(np.r_[v, v[dup], np.zeros(3, np.float32)][perm])
        cols["b"].append(np.r_[base["b"][s:e], base["b"][s:e][dup], extra_b][perm].astype(np.float32))
        sizes.append(e - s + 13)
    offsets = np.zeros(301, np.int64)
    np.cumsum(sizes, out=offsets[1:])
    batch = {k: np.concatenate(v).astype(np.float32) for k, v in cols.items()}
    batch.update({"offsets": offsets, "obj": base["obj"], "box": base["box"]})
    got = gpu_solve3(batch, seed=3, precision=prec)
    ref = oracle3(batch, seed=3)
    assert_parity3(batch, got, ref, TOL[prec])
    assert (ref["status"][::7] == oracle.INFEASIBLE).all()


@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP64])
def test_lps_beyond_the_warp_stage(prec):
    # LPs of 1019 constraints and more run in the one-warp kernel with the large stage;
    # mixed with small ones, 25 % infeasible.  FP64 also takes the oracle's exact path
    # (violation counts).
    sizes = np.array([1019, 2000, 5000, 40, 700, 1019, 2000, 5000, 3, 9000] * 3)
    batch = workloads.sphere_batch(sizes, seed=21, infeasible_frac=0.25)
    want = prec == lp2d.PREC_FP64
    got = gpu_solve3(batch, seed=4, precision=prec, want=want)
    ref = oracle3(batch, seed=4, want_nviol=want)
    assert got["err"] == 0
    assert_parity3(batch, got, ref, TOL[prec])
    if want:
        assert (got["nviol"] == ref["nviol"]).all()


@pytest.mark.parametrize("prec", [lp2d.PREC_FP32, lp2d.PREC_FP64])
def test_hand_solved_degenerate_golden(prec):
    # LPs whose optimum is not a point: the point returned is decided by the frame's
    # orientation (R17), the start's tie rule (R18) and the endpoint rule, and must be
    # the hand-derived one, in both visit orders where the case names one
    import lp_pins

    for case in lp_pins.load_hand_lps_nd():
        if case["solver"] != "3d":
            continue
        seed = 0 if case["order"] is None else lp_pins.seed_for_order(oracle.perm_array, case["order"])
        cons = np.asarray(case["cons"], np.float32)
        batch = {"ax": cons[:, 0].copy(), "ay": cons[:, 1].copy(), "az": cons[:, 2].copy(), "b": cons[:, 3].copy(),
                 "offsets": np.array([0, len(cons)], np.int64), "obj": np.asarray([case["obj"]], np.float32),
                 "box": case["box"]}
        got = gpu_solve3(batch, seed=seed, precision=prec)
        assert got["status"][0] == case["status"], case["name"]
        tol = 1e-12 if prec == lp2d.PREC_FP64 else 1e-6
        assert np.allclose(got["xyz"][0], case["x"], rtol=0, atol=tol), (case["name"], got["xyz"][0])
