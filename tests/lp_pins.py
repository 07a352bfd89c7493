"""Independent checks used to pin the oracle (no code shared with oracle/ or the
CUDA library): hand-solved LP fixtures, brute-force vertex enumeration, and the
LP optimality / infeasibility certificates."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
STATUS = {"OPTIMAL": 0, "INFEASIBLE": 1, "BOX_BOUNDED": 2, "BAD_INPUT": 3}


def load_hand_lps(path=os.path.join(GOLDEN, "hand_lps.txt")):
    """Parse the hand-solved LP fixtures."""
    cases, cur = [], None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "lp":
                cur = {"name": tok[1], "cons": [], "box": None, "obj": None}
                cases.append(cur)
            elif tok[0] == "box":
                cur["box"] = tuple(float(v) for v in tok[1:5])
            elif tok[0] == "obj":
                cur["obj"] = (float(tok[1]), float(tok[2]))
            elif tok[0] == "c":
                cur["cons"].append(tuple(float(v) for v in tok[1:4]))
            elif tok[0] == "expect":
                cur["status"] = STATUS[tok[1]]
                cur["xyf"] = tuple(float(v) for v in tok[2:5]) if len(tok) > 2 else None
    return cases


def load_hand_lps_nd(path=os.path.join(GOLDEN, "hand_lps_nd.txt")):
    """Parse the hand-solved degenerate 3-D and d-dimensional LP fixtures."""
    cases, cur = [], None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "lp":
                cur = {"name": tok[1], "cons": [], "order": None}
                cases.append(cur)
            elif tok[0] == "solver":
                cur["solver"] = tok[1]
            elif tok[0] == "box":
                cur["box"] = tuple(float(v) for v in tok[1:])
            elif tok[0] == "obj":
                cur["obj"] = tuple(float(v) for v in tok[1:])
            elif tok[0] == "c":
                cur["cons"].append(tuple(float(v) for v in tok[1:]))
            elif tok[0] == "order":
                cur["order"] = [int(v) for v in tok[1:]]
            elif tok[0] == "expect":
                cur["status"] = STATUS[tok[1]]
                vals = [float(v) for v in tok[2:]]
                cur["x"], cur["f"] = tuple(vals[:-1]), vals[-1]
    for case in cases:
        d = len(case["obj"])
        assert len(case["box"]) == 2 * d and all(len(c) == d + 1 for c in case["cons"]), case["name"]
        assert case["order"] is None or sorted(case["order"]) == list(range(len(case["cons"]))), case["name"]
    return cases


def seed_for_order(perm_array, order, tries=4096):
    """A seed whose visit order of len(order) constraints is `order` (perm_array(seed,
    m) lists the constraint visited at each position)."""
    for seed in range(tries):
        if list(perm_array(seed, len(order))) == list(order):
            return seed
    raise AssertionError(f"no seed below {tries} gives the visit order {order}")


def box_rows(box):
    """Box sides as (ax, ay, b) rows with ids -1..-4 (x<=xmax, x>=xmin, y<=ymax, y>=ymin)."""
    xmin, xmax, ymin, ymax = box
    return np.array([[1.0, 0.0, xmax], [-1.0, 0.0, -xmin], [0.0, 1.0, ymax], [0.0, -1.0, -ymin]])


def brute_force(ax, ay, b, c, box, feas_tol=1e-9):
    """max c.x over {A x <= b} intersected with the box, by enumerating every vertex.

    Returns (status, xy, f, ids) with status 0/1/2 as in the library (BOX_BOUNDED when
    a box side passes through the best vertex)."""
    rows = np.concatenate([np.stack([ax, ay, b], axis=1).astype(np.float64), box_rows(box)])
    ids = np.concatenate([np.arange(len(ax)), -1 - np.arange(4)])
    n = rows.shape[0]
    ii, jj = np.triu_indices(n, k=1)
    a1, a2 = rows[ii], rows[jj]
    det = a1[:, 0] * a2[:, 1] - a1[:, 1] * a2[:, 0]
    scale = np.hypot(a1[:, 0], a1[:, 1]) * np.hypot(a2[:, 0], a2[:, 1])
    ok = np.abs(det) > 1e-12 * np.maximum(scale, 1e-300)
    ii, jj, a1, a2, det = ii[ok], jj[ok], a1[ok], a2[ok], det[ok]
    x = (a1[:, 2] * a2[:, 1] - a1[:, 1] * a2[:, 2]) / det
    y = (a1[:, 0] * a2[:, 2] - a1[:, 2] * a2[:, 0]) / det
    slack = rows[None, :, 0] * x[:, None] + rows[None, :, 1] * y[:, None] - rows[None, :, 2]
    mag = (np.abs(rows[None, :, 0] * x[:, None]) + np.abs(rows[None, :, 1] * y[:, None])
           + np.abs(rows[None, :, 2]) + 1.0)
    feas = np.all(slack <= feas_tol * mag, axis=1)
    if not feas.any():
        return 1, (np.nan, np.nan), np.nan, None
    f = c[0] * x + c[1] * y
    f[~feas] = -np.inf
    k = int(np.argmax(f))
    pair = (int(ids[ii[k]]), int(ids[jj[k]]))
    # Every line through the best vertex (degenerate vertices have more than two).
    on = np.abs(slack[k]) <= 1e-9 * mag[k]
    through = set(int(v) for v in ids[on])
    status = 2 if any(v < 0 for v in through) else 0
    return status, (x[k], y[k]), f[k], pair


def kkt_certificate(rows_of, xy, c, def_ids, tol=1e-9):
    """Check that xy is optimal: it lies on the two constraints def_ids, satisfies
    every constraint, and c is a non-negative combination of their normals.
    rows_of(id) -> (ax, ay, b) for constraint or box ids; returns the multipliers."""
    i, j = def_ids
    ai, aj = np.array(rows_of(i), float), np.array(rows_of(j), float)
    M = np.array([[ai[0], aj[0]], [ai[1], aj[1]]])
    lam = np.linalg.solve(M, np.asarray(c, float))
    scale = max(1.0, abs(xy[0]), abs(xy[1]))
    for r in (ai, aj):
        assert abs(r[0] * xy[0] + r[1] * xy[1] - r[2]) <= tol * scale * (1 + abs(r[2]))
    assert lam.min() >= -tol * max(1.0, np.abs(lam).max()), lam
    return lam


def farkas_certificate(rows):
    """Check that the 2 or 3 half-planes `rows` (each ax, ay, b) have no common point:
    find y >= 0 with y^T A = 0 and y^T b < 0.  Returns y."""
    R = np.asarray(rows, float)
    if R.shape[0] == 2:
        a, g = R[0], R[1]
        # g's normal must be a negative multiple of a's: g_n = -lam * a_n, lam > 0
        lam = -(g[0] * a[0] + g[1] * a[1]) / (a[0] ** 2 + a[1] ** 2)
        assert lam > 0
        assert abs(g[0] + lam * a[0]) <= 1e-12 * abs(lam) and abs(g[1] + lam * a[1]) <= 1e-12 * abs(lam)
        y = np.array([lam, 1.0])
    else:
        A = R[:, :2]
        # null vector of A^T (2x3): cross products of the columns
        y = np.array([A[1, 0] * A[2, 1] - A[1, 1] * A[2, 0],
                      A[2, 0] * A[0, 1] - A[2, 1] * A[0, 0],
                      A[0, 0] * A[1, 1] - A[0, 1] * A[1, 0]])
        if y.sum() < 0:
            y = -y
        assert y.min() >= -1e-12 * np.abs(y).max(), y
    yb = float(y @ R[:, 2])
    assert yb < 0, (y, R)
    return y


def least_violation_batch(batch, tmax_factor=8.0):
    """The least-violation LP of every LP of a 2-D batch as a 3-D batch in (x, y, t):
    minimise t s.t. a.x - |a| t <= b, (x, y) in the box, 0 <= t <= tmax_factor * max |box|.
    |a| is the float32 value of sqrt(ax*ax + ay*ay) with each operation rounded."""
    ax = np.asarray(batch["ax"], np.float32)
    ay = np.asarray(batch["ay"], np.float32)
    az = -np.sqrt(ax * ax + ay * ay).astype(np.float32)
    box = tuple(float(v) for v in batch["box"])
    tmax = float(np.float32(tmax_factor) * np.float32(max(abs(v) for v in box)))
    n_lp = len(batch["offsets"]) - 1
    obj = np.tile(np.array([0.0, 0.0, -1.0], np.float32), (n_lp, 1))
    return {"ax": ax, "ay": ay, "az": az, "b": np.asarray(batch["b"], np.float32), "offsets": batch["offsets"],
            "obj": obj, "box": box + (0.0, tmax)}

