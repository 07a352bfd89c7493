"""Pins of the 3-D FP64 oracle (oracle/seidel3_oracle.c) to facts that do not come
from the oracle itself: brute-force vertex enumeration, closed forms of regular
polytopes, KKT certificates, the already pinned 2-D oracle on LPs that do not depend
on z, scipy's HiGHS, independence of the visit order and the expected number of
violations of Seidel's method in three dimensions."""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import lp_pins
import oracle
from paper_1902_04995_gb300 import workloads

BOX = workloads.BOX3


def single(a, b, c, box=BOX, seed=0, **kw):
    a = np.asarray(a, np.float32).reshape(-1, 3)
    return oracle.solve_batch3(a[:, 0], a[:, 1], a[:, 2], np.asarray(b, np.float32), np.array([0, a.shape[0]]),
                               np.asarray(c, np.float32).reshape(1, 3), box, seed=seed, **kw)


def box_planes(box):
    xmin, xmax, ymin, ymax, zmin, zmax = box
    a = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
    return a, np.array([xmax, -xmin, ymax, -ymin, zmax, -zmin], np.float64)


def brute_force(a, b, c, box):
    """max c.x over {a x <= b} and the box by enumerating every vertex (triples of
    planes); None when no vertex is feasible."""
    ba, bb = box_planes(box)
    A = np.vstack([np.asarray(a, np.float64).reshape(-1, 3), ba])
    B = np.concatenate([np.asarray(b, np.float64), bb])
    best = None
    for i, j, k in itertools.combinations(range(A.shape[0]), 3):
        M = A[[i, j, k]]
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, B[[i, j, k]])
        if np.all(A @ x <= B + 1e-9 * (np.abs(A) @ np.abs(x) + np.abs(B) + 1.0)):
            f = float(np.dot(c, x))
            best = f if best is None else max(best, f)
    return best


def test_cube_and_box_closed_forms():
    cube = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
    for c in ([1, 2, 3], [-1, 0.5, -2], [0.3, -0.7, 0.1]):
        r = single(cube, np.full(6, 2.0), c, want_def=True)
        assert r["status"][0] == oracle.OPTIMAL
        assert np.allclose(r["xyz"][0], 2.0 * np.sign(c))
        assert r["xyz"][0] @ np.asarray(c, np.float64) == pytest.approx(2.0 * np.abs(c).sum(), rel=1e-12)
    # no constraints: the box corner, box-bounded
    r = oracle.solve_batch3(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                            np.zeros(0, np.float32), np.array([0, 0]), np.array([[1, -1, 1]], np.float32), BOX)
    assert r["status"][0] == oracle.BOX_BOUNDED and np.allclose(r["xyz"][0], [1e3, -1e3, 1e3])


def test_octahedron_closed_form():
    # |x| + |y| + |z| <= 1.5: the optimum of c.x is 1.5 max_j |c_j| at a vertex on an axis
    a = [[sx, sy, sz] for sx in (1, -1) for sy in (1, -1) for sz in (1, -1)]
    for c in ([0.2, -0.9, 0.4], [1.0, 0.3, -0.2], [-0.1, 0.2, -0.8]):
        r = single(a, np.full(8, 1.5), c)
        assert r["status"][0] == oracle.OPTIMAL
        assert r["xyz"][0] @ np.asarray(c, np.float64) == pytest.approx(1.5 * np.abs(c).max(), rel=1e-12)


def test_brute_force_on_tiny_lps():
    rng = np.random.default_rng(33)
    n_inf = 0
    for trial in range(1500):
        m = int(rng.integers(0, 7))
        a = rng.normal(size=(m, 3)).astype(np.float32)
        b = rng.uniform(-1.0, 2.0, size=m).astype(np.float32)
        c = rng.normal(size=3).astype(np.float32)
        box = (-5.0, 5.0, -5.0, 5.0, -5.0, 5.0)
        r = single(a, b, c, box=box, seed=trial)
        ref = brute_force(a, b, c.astype(np.float64), box)
        if ref is None:
            assert r["status"][0] == oracle.INFEASIBLE, trial
            n_inf += 1
        else:
            assert r["status"][0] in (oracle.OPTIMAL, oracle.BOX_BOUNDED), trial
            f = float(r["xyz"][0] @ c.astype(np.float64))
            assert abs(f - ref) <= 1e-9 * max(abs(ref), 1.0), (trial, f, ref)
    assert n_inf > 50  # the sample covers infeasible LPs too


def test_kkt_certificates_on_a_generated_batch():
    batch = workloads.sphere_batch(np.full(400, 60), seed=5, infeasible_frac=0.1)
    r = oracle.solve_batch3(batch["ax"], batch["ay"], batch["az"], batch["b"], batch["offsets"], batch["obj"],
                            batch["box"], seed=9, want_def=True)
    ba, bb = box_planes(batch["box"])
    checked = 0
    for l in range(400):
        s, e = batch["offsets"][l], batch["offsets"][l + 1]
        A = np.stack([batch["ax"][s:e], batch["ay"][s:e], batch["az"][s:e]], 1).astype(np.float64)
        B = batch["b"][s:e].astype(np.float64)
        if r["status"][l] == oracle.INFEASIBLE:
            assert batch["infeasible"][l]
            continue
        x = r["xyz"][l]
        assert np.all(A @ x <= B + 1e-9 * (np.abs(A) @ np.abs(x) + np.abs(B) + 1)), l
        rows = [A[d] if d >= 0 else ba[-1 - d] for d in r["def"][l]]
        lam = np.linalg.solve(np.stack(rows, 1), batch["obj"][l].astype(np.float64))
        assert (lam >= -1e-9).all(), (l, lam)  # c is in the cone of the three active normals
        checked += 1
    assert checked >= 350


def test_reduces_to_the_2d_oracle_when_nothing_depends_on_z():
    batch = workloads.disk_batch(workloads.loguniform_sizes(np.random.default_rng(8), 300, 3, 300), seed=6,
                                 infeasible_frac=0.1)
    zeros = np.zeros_like(batch["ax"])
    obj3 = np.concatenate([batch["obj"], np.zeros((300, 1), np.float32)], 1)
    box3 = tuple(batch["box"]) + (-1e3, 1e3)
    r3 = oracle.solve_batch3(batch["ax"], batch["ay"], zeros, batch["b"], batch["offsets"], obj3, box3, seed=2)
    r2 = oracle.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"], batch["box"], seed=2)
    infeasible = r2["status"] == oracle.INFEASIBLE
    assert np.array_equal(r3["status"] == oracle.INFEASIBLE, infeasible)
    c = batch["obj"].astype(np.float64)
    f2 = np.einsum("ij,ij->i", r2["xy"][~infeasible], c[~infeasible])
    f3 = np.einsum("ij,ij->i", r3["xyz"][~infeasible, :2], c[~infeasible])
    assert np.allclose(f3, f2, rtol=1e-9, atol=1e-9)


def test_scipy_highs_agrees():
    linprog = pytest.importorskip("scipy.optimize").linprog
    batch = workloads.sphere_batch(np.full(60, 50), seed=12, infeasible_frac=0.2)
    r = oracle.solve_batch3(batch["ax"], batch["ay"], batch["az"], batch["b"], batch["offsets"], batch["obj"],
                            batch["box"], seed=0)
    for l in range(60):
        s, e = batch["offsets"][l], batch["offsets"][l + 1]
        A = np.stack([batch["ax"][s:e], batch["ay"][s:e], batch["az"][s:e]], 1).astype(np.float64)
        res = linprog(-batch["obj"][l].astype(np.float64), A_ub=A, b_ub=batch["b"][s:e].astype(np.float64),
                      bounds=[(-1e3, 1e3)] * 3, method="highs")
        if res.status == 2:
            assert r["status"][l] == oracle.INFEASIBLE
        else:
            assert res.status == 0 and r["status"][l] != oracle.INFEASIBLE
            f = float(r["xyz"][l] @ batch["obj"][l].astype(np.float64))
            assert f == pytest.approx(-res.fun, rel=1e-7, abs=1e-7)


def test_result_does_not_depend_on_the_visit_order():
    batch = workloads.sphere_batch(np.full(200, 80), seed=13, infeasible_frac=0.1)
    c = batch["obj"].astype(np.float64)
    ref = None
    for seed in (0, 1, 12345):
        r = oracle.solve_batch3(batch["ax"], batch["ay"], batch["az"], batch["b"], batch["offsets"], batch["obj"],
                                batch["box"], seed=seed)
        f = np.where(r["status"] == oracle.INFEASIBLE, np.nan, np.einsum("ij,ij->i", np.nan_to_num(r["xyz"]), c))
        if ref is None:
            ref = (r["status"].copy(), f)
        else:
            assert np.array_equal(r["status"], ref[0])
            assert np.allclose(f, ref[1], rtol=1e-9, equal_nan=True)


def test_violations_grow_like_three_log_m():
    # In three dimensions the constraint visited at position k (of k+1, plus the box)
    # is violated with probability at most 3 / (k + 1), so E[violations] <= 3 H_m.
    for m in (16, 128, 1024):
        batch = workloads.sphere_batch(np.full(300, m), seed=m)
        r = oracle.solve_batch3(batch["ax"], batch["ay"], batch["az"], batch["b"], batch["offsets"], batch["obj"],
                                batch["box"], seed=1, want_nviol=True, threads=4)
        harmonic = sum(1.0 / k for k in range(1, m + 1))
        assert r["nviol"].mean() <= 3.0 * harmonic + 1.0, (m, r["nviol"].mean())
        assert r["nviol"].mean() >= 0.5 * math.log(m), (m, r["nviol"].mean())


def test_least_violation_closed_form_and_highs():
    import lp_pins

    # x <= -1 and x >= 1: the least violation is 1, at x = 0
    b2 = {"ax": np.array([1, -1], np.float32), "ay": np.array([0, 0], np.float32), "b": np.array([-1, -1], np.float32),
          "offsets": np.array([0, 2]), "obj": np.array([[1, 0]], np.float32), "box": (-10.0, 10.0, -10.0, 10.0)}
    lv = lp_pins.least_violation_batch(b2)
    r = oracle.solve_batch3(lv["ax"], lv["ay"], lv["az"], lv["b"], lv["offsets"], lv["obj"], lv["box"])
    assert r["status"][0] != oracle.INFEASIBLE
    assert r["xyz"][0][0] == pytest.approx(0.0, abs=1e-12) and r["xyz"][0][2] == pytest.approx(1.0, rel=1e-12)
    # infeasible disk-family LPs: the least violation equals HiGHS's minimax value
    linprog = pytest.importorskip("scipy.optimize").linprog
    batch = workloads.disk_batch(np.full(80, 30), seed=21, infeasible_frac=0.5)
    lv = lp_pins.least_violation_batch(batch)
    r = oracle.solve_batch3(lv["ax"], lv["ay"], lv["az"], lv["b"], lv["offsets"], lv["obj"], lv["box"])
    checked = 0
    for l in np.nonzero(batch["infeasible"])[0]:
        s, e = batch["offsets"][l], batch["offsets"][l + 1]
        A = np.stack([lv["ax"][s:e], lv["ay"][s:e], lv["az"][s:e]], 1).astype(np.float64)
        res = linprog([0, 0, 1], A_ub=A, b_ub=lv["b"][s:e].astype(np.float64),
                      bounds=[(-1e3, 1e3), (-1e3, 1e3), (0, lv["box"][5])], method="highs")
        assert res.status == 0
        assert r["xyz"][l][2] == pytest.approx(res.fun, rel=1e-7, abs=1e-7)
        assert r["xyz"][l][2] > 1e-3  # infeasible: some violation is unavoidable
        checked += 1
    assert checked == 40


HAND_3D = [case for case in lp_pins.load_hand_lps_nd() if case["solver"] == "3d"]


@pytest.mark.parametrize("case", HAND_3D, ids=[case["name"] for case in HAND_3D])
def test_hand_solved_degenerate_golden(case):
    # readings R17 (the frame's orientation), R18 (the start's tie rule) and the
    # endpoint rule on a line the objective is orthogonal to, pinned by LPs whose
    # optimum is not a point: the hand-derived optimal point must come back exactly
    seed = 0 if case["order"] is None else lp_pins.seed_for_order(oracle.perm_array, case["order"])
    cons = np.asarray(case["cons"], np.float64)
    r = single(cons[:, :3], cons[:, 3], case["obj"], box=case["box"], seed=seed)
    assert r["status"][0] == case["status"], case["name"]
    assert np.allclose(r["xyz"][0], case["x"], rtol=0, atol=1e-12), (case["name"], r["xyz"][0])
    assert abs(float(np.dot(r["xyz"][0], case["obj"])) - case["f"]) <= 1e-12


def test_every_hand_solved_degenerate_golden():
    for case in HAND_3D:
        test_hand_solved_degenerate_golden(case)
