"""Pins of the d-dimensional FP64 oracle (oracle/seidelN_oracle.c, d <= 5) to facts
that do not come from the oracle itself: brute-force vertex enumeration, closed forms
of the hypercube, cross-polytope and simplex, KKT certificates, the separately pinned
2-D and 3-D oracles, lifting a (d-1)-dimensional LP, scipy's HiGHS, invariance under a
permutation of the axes, independence of the visit order and the expected number of
violations of Seidel's method in d dimensions."""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import lp_pins
import oracle
from paper_1902_04995_gb300 import workloads


def single(a_rows, b, c, box, seed=0, **kw):
    a_rows = np.asarray(a_rows, np.float32).reshape(-1, len(c))
    return oracle.solve_batchN(a_rows.T, np.asarray(b, np.float32), np.array([0, a_rows.shape[0]]),
                               np.asarray(c, np.float32).reshape(1, -1), box, seed=seed, **kw)


def box_planes(box):
    d = len(box) // 2
    a = np.zeros((2 * d, d))
    bb = np.zeros(2 * d)
    for j in range(d):
        a[2 * j, j], bb[2 * j] = 1.0, box[2 * j + 1]
        a[2 * j + 1, j], bb[2 * j + 1] = -1.0, -box[2 * j]
    return a, bb


def brute_force(a_rows, b, c, box):
    """max c.x over {a x <= b} and the box by enumerating every vertex (all d-subsets
    of planes, solved as one stacked system); None when no vertex is feasible."""
    d = len(c)
    ba, bb = box_planes(box)
    A = np.vstack([np.asarray(a_rows, np.float64).reshape(-1, d), ba])
    B = np.concatenate([np.asarray(b, np.float64), bb])
    combos = np.array(list(itertools.combinations(range(A.shape[0]), d)))
    M = A[combos]
    keep = np.abs(np.linalg.det(M)) > 1e-12
    M, R = M[keep], B[combos[keep]]
    X = np.linalg.solve(M, R[..., None])[..., 0]
    slack = X @ A.T - B
    ok = np.all(slack <= 1e-9 * (np.abs(X) @ np.abs(A).T + np.abs(B) + 1.0), axis=1)
    if not ok.any():
        return None
    return float((X[ok] @ np.asarray(c, np.float64)).max())


def objective(r, obj):
    f = np.einsum("ij,ij->i", np.nan_to_num(r["x"]), np.asarray(obj, np.float64))
    return np.where(r["status"] == oracle.INFEASIBLE, np.nan, f)


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_hypercube_cross_polytope_and_simplex_closed_forms(d):
    rng = np.random.default_rng(d)
    box = (-10.0, 10.0) * d
    eye = np.eye(d)
    cube = np.vstack([eye, -eye])
    cross = np.array(list(itertools.product((1.0, -1.0), repeat=d)))
    simplex = np.vstack([-eye, np.ones((1, d))])
    for _ in range(5):
        c = rng.normal(size=d).astype(np.float32)
        c64 = c.astype(np.float64)
        r = single(cube, np.full(2 * d, 2.0), c, box)
        assert r["status"][0] == oracle.OPTIMAL
        assert np.allclose(r["x"][0], 2.0 * np.sign(c64))
        r = single(cross, np.full(2 ** d, 1.5), c, box)
        assert r["status"][0] == oracle.OPTIMAL
        assert r["x"][0] @ c64 == pytest.approx(1.5 * np.abs(c64).max(), rel=1e-12)
        r = single(simplex, np.r_[np.zeros(d), 1.0], c, box)
        assert r["status"][0] == oracle.OPTIMAL
        assert r["x"][0] @ c64 == pytest.approx(max(0.0, c64.max()), abs=1e-12)
    # no constraints: the box corner that maximises c, box-bounded
    c = np.r_[1.0, -1.0, 0.0, 2.0, -3.0][:d].astype(np.float32)
    r = oracle.solve_batchN(np.zeros((d, 0), np.float32), np.zeros(0, np.float32), np.array([0, 0]), c[None],
                            (-3.0, 4.0) * d, want_def=True)
    assert r["status"][0] == oracle.BOX_BOUNDED
    assert np.array_equal(r["x"][0], np.where(c >= 0, 4.0, -3.0))
    assert sorted(r["def"][0]) == sorted(-1 - (2 * j + (c[j] < 0)) for j in range(d))


@pytest.mark.parametrize("d,trials", [(3, 500), (4, 500), (5, 250)])
def test_brute_force_on_tiny_lps(d, trials):
    rng = np.random.default_rng(40 + d)
    box = (-5.0, 5.0) * d
    n_inf = 0
    for trial in range(trials):
        m = int(rng.integers(0, 8 if d < 5 else 7))
        a = rng.normal(size=(m, d)).astype(np.float32)
        b = rng.uniform(-2.0 - 0.5 * (d - 3), 2.0, size=m).astype(np.float32)
        if rng.random() < 0.25:  # a pair of nearly opposite half-spaces with an empty band
            g = rng.normal(size=d)
            beta = rng.uniform(-1.0, 1.0)
            pair = np.stack([g, -g + 0.1 * rng.normal(size=d)])
            a = np.vstack([a, pair]).astype(np.float32)
            b = np.r_[b, beta, -beta - 0.5 * np.linalg.norm(g) - 3.0].astype(np.float32)
            shuffle = rng.permutation(a.shape[0])
            a, b = a[shuffle], b[shuffle]
        c = rng.normal(size=d).astype(np.float32)
        r = single(a, b, c, box, seed=trial)
        ref = brute_force(a, b, c.astype(np.float64), box)
        if ref is None:
            assert r["status"][0] == oracle.INFEASIBLE, trial
            n_inf += 1
        else:
            assert r["status"][0] in (oracle.OPTIMAL, oracle.BOX_BOUNDED), trial
            f = float(r["x"][0] @ c.astype(np.float64))
            assert abs(f - ref) <= 1e-9 * max(abs(ref), 1.0), (trial, f, ref)
    assert n_inf > trials // 20  # the sample covers infeasible LPs too


@pytest.mark.parametrize("d", [4, 5])
def test_kkt_certificates_on_a_generated_batch(d):
    batch = workloads.ball_batch(d, np.full(150, 50), seed=5 + d, infeasible_frac=0.1)
    r = oracle.solve_batchN(batch["a"], batch["b"], batch["offsets"], batch["obj"], batch["box"], seed=9,
                            want_def=True)
    ba, bb = box_planes(batch["box"])
    checked = 0
    for l in range(150):
        s, e = batch["offsets"][l], batch["offsets"][l + 1]
        A = batch["a"][:, s:e].T.astype(np.float64)
        B = batch["b"][s:e].astype(np.float64)
        if r["status"][l] == oracle.INFEASIBLE:
            assert batch["infeasible"][l]
            continue
        assert not batch["infeasible"][l]
        x = r["x"][l]
        assert np.all(A @ x <= B + 1e-9 * (np.abs(A) @ np.abs(x) + np.abs(B) + 1)), l
        assert np.all(ba @ x <= bb + 1e-9 * (np.abs(ba) @ np.abs(x) + np.abs(bb) + 1)), l
        rows = [A[q] if q >= 0 else ba[-1 - q] for q in r["def"][l]]
        rhs = [B[q] if q >= 0 else bb[-1 - q] for q in r["def"][l]]
        N = np.stack(rows)
        assert np.allclose(N @ x, rhs, rtol=1e-9, atol=1e-9), l  # the d defining planes are tight
        lam = np.linalg.solve(N.T, batch["obj"][l].astype(np.float64))
        assert (lam >= -1e-9).all(), (l, lam)  # c is in the cone of the d active normals
        checked += 1
    assert checked >= 120


def test_agrees_with_the_2d_and_3d_oracles():
    sizes = workloads.loguniform_sizes(np.random.default_rng(8), 300, 3, 300)
    b2 = workloads.disk_batch(sizes, seed=6, infeasible_frac=0.1)
    r2 = oracle.solve_batch(b2["ax"], b2["ay"], b2["b"], b2["offsets"], b2["obj"], b2["box"], seed=2)
    rn = oracle.solve_batchN(np.stack([b2["ax"], b2["ay"]]), b2["b"], b2["offsets"], b2["obj"], b2["box"], seed=2)
    assert np.array_equal(rn["status"] == oracle.INFEASIBLE, r2["status"] == oracle.INFEASIBLE)
    f2 = objective({"x": r2["xy"], "status": r2["status"]}, b2["obj"])
    assert np.allclose(objective(rn, b2["obj"]), f2, rtol=1e-9, atol=1e-9, equal_nan=True)
    b3 = workloads.sphere_batch(sizes, seed=7, infeasible_frac=0.1)
    r3 = oracle.solve_batch3(b3["ax"], b3["ay"], b3["az"], b3["b"], b3["offsets"], b3["obj"], b3["box"], seed=4)
    rn = oracle.solve_batchN(np.stack([b3["ax"], b3["ay"], b3["az"]]), b3["b"], b3["offsets"], b3["obj"],
                             b3["box"], seed=4)
    assert np.array_equal(rn["status"] == oracle.INFEASIBLE, r3["status"] == oracle.INFEASIBLE)
    f3 = objective({"x": r3["xyz"], "status": r3["status"]}, b3["obj"])
    assert np.allclose(objective(rn, b3["obj"]), f3, rtol=1e-9, atol=1e-9, equal_nan=True)


@pytest.mark.parametrize("d", [4, 5])
def test_lifting_a_lower_dimensional_lp(d):
    # constraints that do not involve the last axis and an objective without it: the
    # optimum is the (d-1)-dimensional one, whatever the last coordinate
    low = workloads.ball_batch(d - 1, workloads.loguniform_sizes(np.random.default_rng(d), 120, 4, 120), seed=d,
                               infeasible_frac=0.15)
    n = low["a"].shape[1]
    a = np.vstack([low["a"], np.zeros((1, n), np.float32)])
    obj = np.hstack([low["obj"], np.zeros((120, 1), np.float32)])
    box = tuple(low["box"]) + (-7.0, 3.0)
    r_low = oracle.solve_batchN(low["a"], low["b"], low["offsets"], low["obj"], low["box"], seed=1)
    r = oracle.solve_batchN(a, low["b"], low["offsets"], obj, box, seed=1)
    assert np.array_equal(r["status"] == oracle.INFEASIBLE, r_low["status"] == oracle.INFEASIBLE)
    assert np.allclose(objective(r, obj), objective(r_low, low["obj"]), rtol=1e-9, atol=1e-9, equal_nan=True)


@pytest.mark.parametrize("d", [4, 5])
def test_scipy_highs_agrees(d):
    linprog = pytest.importorskip("scipy.optimize").linprog
    batch = workloads.ball_batch(d, np.full(50, 40), seed=12 + d, infeasible_frac=0.2)
    r = oracle.solve_batchN(batch["a"], batch["b"], batch["offsets"], batch["obj"], batch["box"], seed=0)
    for l in range(50):
        s, e = batch["offsets"][l], batch["offsets"][l + 1]
        res = linprog(-batch["obj"][l].astype(np.float64), A_ub=batch["a"][:, s:e].T.astype(np.float64),
                      b_ub=batch["b"][s:e].astype(np.float64), bounds=[(-1e3, 1e3)] * d, method="highs")
        if res.status == 2:
            assert r["status"][l] == oracle.INFEASIBLE
        else:
            assert res.status == 0 and r["status"][l] != oracle.INFEASIBLE
            f = float(r["x"][l] @ batch["obj"][l].astype(np.float64))
            assert f == pytest.approx(-res.fun, rel=1e-7, abs=1e-7)


@pytest.mark.parametrize("d", [4, 5])
def test_permuting_the_axes(d):
    batch = workloads.ball_batch(d, np.full(100, 30), seed=30 + d, infeasible_frac=0.1)
    box = tuple(float(v) for v in np.arange(1, 2 * d + 1) * np.tile([-10.0, 7.0], d))
    perm = np.random.default_rng(d).permutation(d)
    boxp = tuple(v for j in perm for v in box[2 * j:2 * j + 2])
    r = oracle.solve_batchN(batch["a"], batch["b"], batch["offsets"], batch["obj"], box, seed=3)
    rp = oracle.solve_batchN(batch["a"][perm], batch["b"], batch["offsets"], batch["obj"][:, perm], boxp, seed=3)
    assert np.array_equal(r["status"], rp["status"])
    ok = r["status"] != oracle.INFEASIBLE
    assert np.allclose(rp["x"][ok], r["x"][ok][:, perm], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("d", [4, 5])
def test_result_does_not_depend_on_the_visit_order(d):
    batch = workloads.ball_batch(d, np.full(100, 60), seed=13, infeasible_frac=0.1)
    ref = None
    for seed in (0, 1, 12345):
        r = oracle.solve_batchN(batch["a"], batch["b"], batch["offsets"], batch["obj"], batch["box"], seed=seed)
        f = objective(r, batch["obj"])
        if ref is None:
            ref = (r["status"].copy(), f)
        else:
            assert np.array_equal(r["status"], ref[0])
            assert np.allclose(f, ref[1], rtol=1e-9, equal_nan=True)


@pytest.mark.parametrize("d", [4, 5])
def test_violations_grow_like_d_log_m(d):
    # the constraint visited at position k is violated with probability at most
    # d / (k + 1) (the optimum of the first k + 1 is fixed by d of them), so
    # E[violations] <= d H_m
    for m in (16, 128):
        batch = workloads.ball_batch(d, np.full(100, m), seed=m + d)
        r = oracle.solve_batchN(batch["a"], batch["b"], batch["offsets"], batch["obj"], batch["box"], seed=1,
                                want_nviol=True, threads=4)
        harmonic = sum(1.0 / k for k in range(1, m + 1))
        assert r["nviol"].mean() <= d * harmonic + 1.0, (m, r["nviol"].mean())
        assert r["nviol"].mean() >= 0.5 * math.log(m), (m, r["nviol"].mean())


def test_bad_input_and_zero_normals():
    d = 4
    box = (-1.0, 1.0) * d
    # a NaN coefficient: BAD_INPUT
    r = single([[np.nan, 0, 0, 0]], [1.0], [1, 0, 0, 0], box)
    assert r["status"][0] == oracle.BAD_INPUT and np.isnan(r["x"][0]).all()
    # 0.x <= -1 excludes everything; 0.x <= 1 excludes nothing
    r = single([[0, 0, 0, 0], [1, 1, 0, 0]], [-1.0, 0.5], [1, 1, 1, 1], box)
    assert r["status"][0] == oracle.INFEASIBLE
    r = single([[0, 0, 0, 0], [1, 1, 0, 0]], [1.0, 0.5], [1, 1, 1, 1], box)
    assert r["status"][0] == oracle.BOX_BOUNDED
    assert r["x"][0] @ np.ones(4) == pytest.approx(2.5, rel=1e-12)


HAND_ND = [case for case in lp_pins.load_hand_lps_nd() if case["solver"] == "nd"]


@pytest.mark.parametrize("case", HAND_ND, ids=[case["name"] for case in HAND_ND])
def test_hand_solved_degenerate_golden(case):
    # the tie rules of R23 (the pivot) and R24 (the start) and the endpoint rule on a
    # line the objective is orthogonal to, pinned by LPs whose optimum is not a point
    seed = 0 if case["order"] is None else lp_pins.seed_for_order(oracle.perm_array, case["order"])
    cons = np.asarray(case["cons"], np.float64)
    d = len(case["obj"])
    r = single(cons[:, :d], cons[:, d], case["obj"], case["box"], seed=seed)
    assert r["status"][0] == case["status"], case["name"]
    assert np.allclose(r["x"][0], case["x"], rtol=0, atol=1e-12), (case["name"], r["x"][0])
    assert abs(float(np.dot(r["x"][0], case["obj"])) - case["f"]) <= 1e-12


def test_every_hand_solved_degenerate_golden():
    for case in HAND_ND:
        test_hand_solved_degenerate_golden(case)
