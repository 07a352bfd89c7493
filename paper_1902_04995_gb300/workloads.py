"""Seeded synthetic LP batches (the only module shared by the CUDA path's callers
and the oracle's tests).

It holds none of the solver's arithmetic: it draws random constraint sets with
numpy's PCG64 (``default_rng``) and lays them out as the library expects:

* ``ax, ay, b``  float32 [n_constraints]   constraint i is  ax[i]*x + ay[i]*y <= b[i]
* ``offsets``    int64  [n_lp + 1]         LP l owns constraints offsets[l] .. offsets[l+1]-1
* ``obj``        float32 [n_lp, 2]         objective (c_x, c_y) per LP, maximised
* ``box``        (xmin, xmax, ymin, ymax)  the bounding constraints (+-M, Sec. 2.1)

The paper generates random feasible 2-D constraint sets (Sec. 4); these generators
stand in for that, with distinct LPs instead of one LP copied across the batch.

"Disk" family (the plain, at-scale and ragged workloads):
  per LP a centre c ~ U[-1,1]^2; per constraint a unit normal n at angle ~ U[0, 2pi),
  r ~ U[0.5, 2] and b = r + n.c, so c is strictly feasible (margin >= 0.5) and every
  LP is feasible; the objective is a unit vector at angle ~ U[0, 2pi).
  A fraction of LPs is made infeasible by appending one constraint  -u.x <= -(H + 1),
  where H >= max over the feasible polygon of u.x.  H comes from weak duality: u is
  written as alpha*n_i + beta*n_j (alpha, beta >= 0) with n_i, n_j the stored normals
  that bracket u in angle, so u.x <= alpha*b_i + beta*b_j for every feasible x.
  Directions whose bracketing gap is >= pi (polygon unbounded there) are redrawn.

Collision-avoidance family (the precision workload):
  a 16-gon of inradius R ~ U[1, 2] around the origin (normals at 2*pi*k/16) plus
  K ~ U{10..100} neighbour half-planes with normal p/|p|, p ~ U[-5,5]^2 and offset
  ~ U[0, 0.5]; 5 % of neighbour normals are replaced by a copy of an earlier normal
  of the same LP rotated by delta ~ U(-1e-6, 1e-6) rad (near-parallel pairs).  The
  origin is feasible in every LP; the objective is a unit preferred-velocity direction.

Sphere family (the 3-D workloads; constraint i is ax[i] x + ay[i] y + az[i] z <= b[i],
``obj`` is [n_lp, 3] and ``box`` has six entries):
  per LP a centre c ~ U[-1,1]^3; per constraint a unit normal n uniform on the sphere
  (a normalised Gaussian), r ~ U[0.5, 2] and b = r + n.c, so the ball of radius 0.5
  around c is feasible; the objective is a unit vector uniform on the sphere.  An LP
  is made infeasible with  -u.x <= -(H + 1),  H = sum of lambda_k b_k over three stored
  normals with u = sum lambda_k n_k, lambda >= 0 (weak duality bounds u.x by H).

Ball family (d = 2..5 dimensions; ``a`` is float32 [d, n_constraints], row t holding
coefficient t of every constraint, ``obj`` is [n_lp, d] and ``box`` has 2d entries):
  the sphere family in d dimensions: centre c ~ U[-1,1]^d, unit normals uniform on the
  sphere, r ~ U[0.5, 2], b = r + n.c, unit objective uniform on the sphere.  An LP is
  made infeasible with  -u.x <= -(H + 1)  for u = sum_k lambda_k n_k / |.| over d
  distinct stored normals drawn at random, lambda_k ~ U[0.1, 1] and
  H = sum_k lambda_k b_k / |sum_k lambda_k n_k| (weak duality bounds u.x by H).
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20190213
BOX_M = 1e3
DEFAULT_BOX = (-BOX_M, BOX_M, -BOX_M, BOX_M)


def _disk_constraints(rng, sizes):
    """Constraints of the disk family for LPs of the given sizes (float32 SoA)."""
    n_lp = sizes.shape[0]
    offsets = np.zeros(n_lp + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    centre = rng.uniform(-1.0, 1.0, size=(n_lp, 2))
    theta = rng.uniform(0.0, 2.0 * math.pi, size=total)
    r = rng.uniform(0.5, 2.0, size=total)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n_lp)
    owner = np.repeat(np.arange(n_lp, dtype=np.int64), sizes)
    nx = np.cos(theta)
    ny = np.sin(theta)
    del theta
    b = r + nx * centre[owner, 0] + ny * centre[owner, 1]
    del r, owner
    obj = np.stack([np.cos(phi), np.sin(phi)], axis=1).astype(np.float32)
    return (nx.astype(np.float32), ny.astype(np.float32), b.astype(np.float32), offsets, obj, centre)


def _exclusion_constraint(rng, nx, ny, b):
    """One constraint (a_x, a_y, b) that no point of {n_i . x <= b_i} satisfies.

    nx, ny, b: the LP's stored float32 constraints.  Returns float32 values."""
    nx64 = nx.astype(np.float64)
    ny64 = ny.astype(np.float64)
    b64 = b.astype(np.float64)
    ang = np.arctan2(ny64, nx64)
    order = np.argsort(ang, kind="stable")
    sang = ang[order]
    m = sang.shape[0]
    for attempt in range(65):
        if attempt < 64:
            psi = rng.uniform(-math.pi, math.pi)
        else:  # fall back to the middle of the narrowest gap
            gaps = np.diff(np.concatenate([sang, sang[:1] + 2 * math.pi]))
            g = int(np.argmin(gaps))
            psi = sang[g] + 0.5 * gaps[g]
            psi = (psi + math.pi) % (2 * math.pi) - math.pi
        k = int(np.searchsorted(sang, psi, side="right"))
        i = order[(k - 1) % m]
        j = order[k % m]
        gap = (ang[j] - ang[i]) % (2 * math.pi)
        if m == 1 or gap >= math.pi - 1e-9:
            continue
        ux, uy = math.cos(psi), math.sin(psi)
        det = nx64[i] * ny64[j] - ny64[i] * nx64[j]
        if det == 0.0:
            if abs(nx64[i] * ux + ny64[i] * uy - 1.0) > 1e-12:
                continue
            alpha, beta = 1.0, 0.0
        else:
            alpha = (ux * ny64[j] - uy * nx64[j]) / det
            beta = (nx64[i] * uy - ny64[i] * ux) / det
        if alpha < 0.0 or beta < 0.0:
            continue
        h = alpha * b64[i] + beta * b64[j]
        return np.float32(-ux), np.float32(-uy), np.float32(-(h + 1.0))
    raise RuntimeError("no bounded direction found for the exclusion constraint")


def disk_batch(sizes, seed=DEFAULT_SEED, infeasible_frac=0.0, box=DEFAULT_BOX):
    """A batch of disk-family LPs with the given constraint counts.

    A fraction ``infeasible_frac`` of the LPs (round(frac * n_lp), chosen by a seeded
    sample among the LPs with at least 3 constraints, where a bounded direction always
    exists) gets one appended exclusion constraint, so their size is sizes[l] + 1."""
    sizes = np.asarray(sizes, dtype=np.int64)
    rng = np.random.default_rng(seed)
    ax, ay, b, offsets, obj, _centre = _disk_constraints(rng, sizes)
    n_lp = sizes.shape[0]
    eligible = np.nonzero(sizes >= 3)[0]
    n_inf = min(int(round(infeasible_frac * n_lp)), eligible.shape[0])
    infeasible = np.zeros(n_lp, dtype=bool)
    if n_inf > 0:
        pick = np.sort(eligible[rng.choice(eligible.shape[0], size=n_inf, replace=False)])
        infeasible[pick] = True
        extra = np.zeros((n_inf, 3), dtype=np.float32)
        for t, l in enumerate(pick):
            s, e = offsets[l], offsets[l + 1]
            extra[t] = _exclusion_constraint(rng, ax[s:e], ay[s:e], b[s:e])
        new_sizes = sizes + infeasible.astype(np.int64)
        new_off = np.zeros(n_lp + 1, dtype=np.int64)
        np.cumsum(new_sizes, out=new_off[1:])
        total = int(new_off[-1])
        # Destination of each original constraint: shift by the number of extra
        # slots inserted before its LP.
        shift = np.repeat(new_off[:-1] - offsets[:-1], sizes)
        dst = np.arange(offsets[-1], dtype=np.int64) + shift
        del shift
        nax = np.empty(total, np.float32)
        nay = np.empty(total, np.float32)
        nb = np.empty(total, np.float32)
        nax[dst] = ax
        nay[dst] = ay
        nb[dst] = b
        del dst
        slot = new_off[pick + 1] - 1
        nax[slot] = extra[:, 0]
        nay[slot] = extra[:, 1]
        nb[slot] = extra[:, 2]
        ax, ay, b, offsets = nax, nay, nb, new_off
    return {
        "ax": ax, "ay": ay, "b": b, "offsets": offsets, "obj": obj,
        "box": tuple(float(v) for v in box), "infeasible": infeasible,
    }


def loguniform_sizes(rng, n_lp, lo, hi):
    """floor(exp(U[ln lo, ln(hi + 1)))) -- integer sizes log-uniform over [lo, hi]."""
    s = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size=n_lp))).astype(np.int64)
    return np.clip(s, lo, hi)


def collision_batch(n_lp, seed=DEFAULT_SEED, near_parallel_frac=0.05, box=DEFAULT_BOX):
    """Collision-avoidance-shaped LPs (16-gon speed limit + neighbour half-planes)."""
    rng = np.random.default_rng(seed)
    k_nb = rng.integers(10, 101, size=n_lp)
    sizes = 16 + k_nb
    offsets = np.zeros(n_lp + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    ax = np.empty(total, np.float64)
    ay = np.empty(total, np.float64)
    b = np.empty(total, np.float64)
    radius = rng.uniform(1.0, 2.0, size=n_lp)
    gon = 2.0 * math.pi * np.arange(16) / 16.0
    pref = rng.uniform(0.0, 2.0 * math.pi, size=n_lp)
    for l in range(n_lp):
        s = int(offsets[l])
        k = int(k_nb[l])
        ax[s:s + 16] = np.cos(gon)
        ay[s:s + 16] = np.sin(gon)
        b[s:s + 16] = radius[l]
        p = rng.uniform(-5.0, 5.0, size=(k, 2))
        nrm = np.linalg.norm(p, axis=1)
        nrm[nrm == 0.0] = 1.0
        ang = np.arctan2(p[:, 1] / nrm, p[:, 0] / nrm)
        near = rng.random(k) < near_parallel_frac
        for t in np.nonzero(near)[0]:
            # an earlier constraint of this LP (polygon side or earlier neighbour)
            src = int(rng.integers(0, 16 + t))
            base = gon[src] if src < 16 else ang[src - 16]
            ang[t] = base + rng.uniform(-1e-6, 1e-6)
        ax[s + 16:s + 16 + k] = np.cos(ang)
        ay[s + 16:s + 16 + k] = np.sin(ang)
        b[s + 16:s + 16 + k] = rng.uniform(0.0, 0.5, size=k)
    obj = np.stack([np.cos(pref), np.sin(pref)], axis=1).astype(np.float32)
    return {
        "ax": ax.astype(np.float32), "ay": ay.astype(np.float32), "b": b.astype(np.float32),
        "offsets": offsets, "obj": obj, "box": tuple(float(v) for v in box),
        "infeasible": np.zeros(n_lp, dtype=bool),
    }


# ----------------------------------------------------------------- named workloads
def near_parallel_pairs(n_lp=4096, seed=DEFAULT_SEED, delta=1e-5, margin=1e-3, half=1000.0, tilt=-0.5):
    """LPs whose outcome is the intersection of two nearly parallel lines.

    LP l holds n1 . x <= 0 and n2 . x >= w (stored as -n2 . x <= -w), where n1 has a
    uniform angle and n2 is n1 turned by an angle of delta * U[0.5, 2].  The lines
    cross on the line n1 . x = 0 at s* = w / det(n1, n2) along u = (-n1_y, n1_x); w
    puts that crossing a fraction `margin` inside (even l) or outside (odd l) the box
    of half-width `half`, so the LP is feasible with its optimum at the crossing, or
    infeasible.  The objective n1 + tilt * u makes both visit orders end in the 1-D LP
    on one of the two lines with the other as its bound, where the crossing is the
    quotient of two quantities about delta small: FP32 resolves it only to about
    2^-24 / delta relative, FP64 to about 2^-53 / delta.  Every quantity is computed
    from the float32 values actually stored."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 2.0 * np.pi, n_lp)
    d = delta * rng.uniform(0.5, 2.0, n_lp)
    n1 = np.stack([np.cos(a), np.sin(a)], 1).astype(np.float32)
    n2 = np.stack([np.cos(a + d), np.sin(a + d)], 1).astype(np.float32)
    n1d, n2d = n1.astype(np.float64), n2.astype(np.float64)
    det = n1d[:, 0] * n2d[:, 1] - n1d[:, 1] * n2d[:, 0]
    u = np.stack([-n1d[:, 1], n1d[:, 0]], 1)
    f = np.where(np.arange(n_lp) % 2 == 0, 1.0 - margin, 1.0 + margin)
    w = (f * half * det / np.abs(u).max(1)).astype(np.float32)
    cons = np.zeros((n_lp, 2, 3), np.float32)
    cons[:, 0, :2] = n1
    cons[:, 1, :2] = -n2
    cons[:, 1, 2] = -w
    cons = cons.reshape(-1, 3)
    return {"ax": cons[:, 0].copy(), "ay": cons[:, 1].copy(), "b": cons[:, 2].copy(),
            "offsets": np.arange(0, 2 * n_lp + 1, 2, dtype=np.int64),
            "obj": (n1d + tilt * u).astype(np.float32), "box": (-half, half, -half, half)}


def plain_small(seed=DEFAULT_SEED):
    """256 LPs x 64 constraints, all feasible."""
    return disk_batch(np.full(256, 64, dtype=np.int64), seed=seed)


def plain_at_scale(seed=DEFAULT_SEED, n_lp=65536, m=256):
    """65,536 LPs x 256 constraints; 10 % get a 257th constraint that makes them infeasible."""
    return disk_batch(np.full(n_lp, m, dtype=np.int64), seed=seed, infeasible_frac=0.1)


def ragged(seed=DEFAULT_SEED, n_lp=131072, lo=8, hi=2048):
    """131,072 LPs with sizes log-uniform in [8, 2048]; 10 % infeasible."""
    size_rng = np.random.default_rng(seed ^ 0x5EED5EED)
    sizes = loguniform_sizes(size_rng, n_lp, lo, hi)
    return disk_batch(sizes, seed=seed, infeasible_frac=0.1)


def collision(seed=DEFAULT_SEED, n_lp=16384):
    """16,384 collision-avoidance LPs with 5 % near-parallel neighbour constraints."""
    return collision_batch(n_lp, seed=seed)


def serving_pool(seed=DEFAULT_SEED, n_lp=65536, lo_m=16, hi_m=4096):
    """LPs that resident serving requests draw their ranges from: sizes log-uniform
    in [lo_m, hi_m] as in serving_request, disk family, 10 % infeasible."""
    rng = np.random.default_rng(seed)
    return disk_batch(loguniform_sizes(rng, n_lp, lo_m, hi_m), seed=seed, infeasible_frac=0.1)


def serving_request(seed, lo_lp=1024, hi_lp=65536, lo_m=16, hi_m=4096):
    """One serving request: log-uniform [1k, 64k] LPs with sizes log-uniform in
    [16, 4096], the ragged generator, 10 % infeasible."""
    rng = np.random.default_rng(seed ^ 0xA11CE)
    n_lp = int(loguniform_sizes(rng, 1, lo_lp, hi_lp)[0])
    sizes = loguniform_sizes(rng, n_lp, lo_m, hi_m)
    return disk_batch(sizes, seed=seed, infeasible_frac=0.1)


BOX3 = (-BOX_M, BOX_M, -BOX_M, BOX_M, -BOX_M, BOX_M)


def _exclusion_plane(rng, n, b):
    """One plane (a, b) that no point of {n_i . x <= b_i} satisfies (3-D).

    n: [m, 3] stored float32 normals, b: [m] offsets.  Returns float32 values."""
    n64 = n.astype(np.float64)
    b64 = b.astype(np.float64)
    for _ in range(64):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        near = np.argsort(-(n64 @ u), kind="stable")[:8]
        for i in range(len(near)):
            for j in range(i + 1, len(near)):
                for k in range(j + 1, len(near)):
                    cone = n64[[near[i], near[j], near[k]]].T
                    if abs(np.linalg.det(cone)) < 1e-9:
                        continue
                    lam = np.linalg.solve(cone, u)
                    if (lam >= 0.0).all():
                        h = float(lam @ b64[[near[i], near[j], near[k]]])
                        return np.float32(-u[0]), np.float32(-u[1]), np.float32(-u[2]), np.float32(-(h + 1.0))
    raise RuntimeError("no bounded direction found for the exclusion plane")


def sphere_batch(sizes, seed=DEFAULT_SEED, infeasible_frac=0.0, box=BOX3):
    """A batch of 3-D sphere-family LPs with the given constraint counts.

    A fraction ``infeasible_frac`` of the LPs (chosen by a seeded sample among those
    with at least 8 constraints) gets one appended exclusion plane."""
    sizes = np.asarray(sizes, dtype=np.int64)
    rng = np.random.default_rng(seed)
    n_lp = sizes.shape[0]
    offsets = np.zeros(n_lp + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    centre = rng.uniform(-1.0, 1.0, size=(n_lp, 3))
    nrm = rng.normal(size=(total, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r = rng.uniform(0.5, 2.0, size=total)
    owner = np.repeat(np.arange(n_lp), sizes)
    bb = r + np.einsum("ij,ij->i", nrm, centre[owner])
    obj = rng.normal(size=(n_lp, 3))
    obj /= np.linalg.norm(obj, axis=1, keepdims=True)
    n32 = nrm.astype(np.float32)
    b32 = bb.astype(np.float32)
    eligible = np.nonzero(sizes >= 8)[0]
    n_inf = min(int(round(infeasible_frac * n_lp)), eligible.shape[0])
    infeasible = np.zeros(n_lp, dtype=bool)
    extra = {}
    if n_inf > 0:
        pick = np.sort(eligible[rng.choice(eligible.shape[0], size=n_inf, replace=False)])
        infeasible[pick] = True
        for l in pick:
            s, e = offsets[l], offsets[l + 1]
            extra[int(l)] = _exclusion_plane(rng, n32[s:e], b32[s:e])
    new_sizes = sizes + infeasible.astype(np.int64)
    new_off = np.zeros(n_lp + 1, dtype=np.int64)
    np.cumsum(new_sizes, out=new_off[1:])
    dst = np.arange(total, dtype=np.int64) + np.repeat(new_off[:-1] - offsets[:-1], sizes)
    out = {k: np.empty(int(new_off[-1]), np.float32) for k in ("ax", "ay", "az", "b")}
    for k, col in (("ax", n32[:, 0]), ("ay", n32[:, 1]), ("az", n32[:, 2]), ("b", b32)):
        out[k][dst] = col
    for l, (px, py, pz, pb) in extra.items():
        slot = new_off[l + 1] - 1
        out["ax"][slot], out["ay"][slot], out["az"][slot], out["b"][slot] = px, py, pz, pb
    out.update({"offsets": new_off, "obj": obj.astype(np.float32), "box": tuple(float(v) for v in box),
                "infeasible": infeasible})
    return out


def plain3d(seed=DEFAULT_SEED, n_lp=65536, m=128):
    """65,536 3-D LPs x 128 constraints; 10 % get a 129th that makes them infeasible."""
    return sphere_batch(np.full(n_lp, m, dtype=np.int64), seed=seed, infeasible_frac=0.1)


def ragged3d(seed=DEFAULT_SEED, n_lp=65536, lo=8, hi=1017):
    """65,536 3-D LPs with sizes log-uniform in [8, 1017]; 10 % get one more
    constraint (at most 1018, the 3-D solver's stage capacity) that makes them
    infeasible."""
    size_rng = np.random.default_rng(seed ^ 0x3D3D3D)
    sizes = loguniform_sizes(size_rng, n_lp, lo, hi)
    return sphere_batch(sizes, seed=seed, infeasible_frac=0.1)


def ball_batch(d, sizes, seed=DEFAULT_SEED, infeasible_frac=0.0, box=None):
    """A batch of d-dimensional ball-family LPs with the given constraint counts.

    A fraction ``infeasible_frac`` of the LPs (a seeded sample among those with at
    least max(8, d) constraints) gets one appended exclusion constraint."""
    sizes = np.asarray(sizes, dtype=np.int64)
    box = tuple(float(v) for v in (box if box is not None else (-BOX_M, BOX_M) * d))
    assert 1 <= d <= 5 and len(box) == 2 * d
    rng = np.random.default_rng(seed)
    n_lp = sizes.shape[0]
    offsets = np.zeros(n_lp + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    centre = rng.uniform(-1.0, 1.0, size=(n_lp, d))
    nrm = rng.normal(size=(total, d))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r = rng.uniform(0.5, 2.0, size=total)
    owner = np.repeat(np.arange(n_lp), sizes)
    bb = r + np.einsum("ij,ij->i", nrm, centre[owner])
    obj = rng.normal(size=(n_lp, d))
    obj /= np.linalg.norm(obj, axis=1, keepdims=True)
    n32 = nrm.astype(np.float32)
    b32 = bb.astype(np.float32)
    eligible = np.nonzero(sizes >= max(8, d))[0]
    n_inf = min(int(round(infeasible_frac * n_lp)), eligible.shape[0])
    infeasible = np.zeros(n_lp, dtype=bool)
    extra = {}
    if n_inf > 0:
        pick = np.sort(eligible[rng.choice(eligible.shape[0], size=n_inf, replace=False)])
        infeasible[pick] = True
        for l in pick:
            s = offsets[l]
            idx = s + rng.choice(int(sizes[l]), size=d, replace=False)
            lam = rng.uniform(0.1, 1.0, size=d)
            u = lam @ n32[idx].astype(np.float64)
            h = float(lam @ b32[idx].astype(np.float64))
            nu = float(np.linalg.norm(u))
            extra[int(l)] = ((-u / nu).astype(np.float32), np.float32(-(h / nu + 1.0)))
    new_sizes = sizes + infeasible.astype(np.int64)
    new_off = np.zeros(n_lp + 1, dtype=np.int64)
    np.cumsum(new_sizes, out=new_off[1:])
    dst = np.arange(total, dtype=np.int64) + np.repeat(new_off[:-1] - offsets[:-1], sizes)
    a = np.empty((d, int(new_off[-1])), np.float32)
    bo = np.empty(int(new_off[-1]), np.float32)
    a[:, dst] = n32.T
    bo[dst] = b32
    for l, (pa, pb) in extra.items():
        slot = new_off[l + 1] - 1
        a[:, slot] = pa
        bo[slot] = pb
    return {"a": a, "b": bo, "offsets": new_off, "obj": obj.astype(np.float32), "box": box,
            "infeasible": infeasible}


def ragged_nd(d, seed=DEFAULT_SEED, n_lp=65536, lo=8, hi=None):
    """65,536 ball-family LPs in d dimensions with sizes log-uniform in [8, hi]
    (default 1023 - 2d, so that with the appended constraint of the 10 % made
    infeasible no LP exceeds the d-dimensional solver's 1024 - 2d)."""
    hi = 1023 - 2 * d if hi is None else hi
    size_rng = np.random.default_rng(seed ^ (0xD0D0 + d))
    sizes = loguniform_sizes(size_rng, n_lp, lo, hi)
    return ball_batch(d, sizes, seed=seed, infeasible_frac=0.1)


WORKLOADS = {
    "plain_small_256x64": plain_small,
    "plain_65536x256": plain_at_scale,
    "ragged_131072_logu8_2048": ragged,
    "collision_16384": collision,
}


def algorithmic_bytes(batch) -> int:
    """Bytes one solve must move at minimum: 12 B per constraint read once, plus per
    LP 8 B objective, 8 B offset, 8 B result point and 4 B status (3-D: 16 B per
    constraint and 12 + 8 + 12 + 4 B per LP; d dimensions: 4d + 4 B per constraint and
    4d + 8 + 4d + 4 B per LP)."""
    n_c = int(batch["offsets"][-1] - batch["offsets"][0])
    n_lp = int(batch["offsets"].shape[0] - 1)
    if "a" in batch:
        d = int(batch["a"].shape[0])
        return (4 * d + 4) * n_c + (8 * d + 12) * n_lp
    if "az" in batch:
        return 16 * n_c + 36 * n_lp
    return 12 * n_c + 28 * n_lp
