"""Pins of the FP64 oracle against things other than itself: hand-solved LPs, brute
force vertex enumeration, closed forms, LP certificates, a published PRNG test
vector, permutation invariants and a library LP solver.  CPU only."""
from __future__ import annotations

import math

import numpy as np
import pytest

import lp_pins
from paper_1902_04995_gb300 import workloads

BOX = (-1e3, 1e3, -1e3, 1e3)


def solve_one(oracle, cons, c, box=BOX, seed=0):
    cons = np.asarray(cons, dtype=np.float32).reshape(-1, 3)
    off = np.array([0, cons.shape[0]], dtype=np.int64)
    r = oracle.solve_batch(cons[:, 0], cons[:, 1], cons[:, 2], off, np.asarray(c, np.float32), box,
                           seed=seed, want_def=True, want_nviol=True)
    return r["status"][0], r["xy"][0], r["def"][0], r["nviol"][0]


# ----------------------------------------------------------- visit order pi
def test_splitmix64_published_vector(oracle_mod):
    # Reference output of SplitMix64 (Steele, Lea & Flood 2014; Vigna's splitmix64.c)
    # for seed 1234567: the first five outputs.
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    assert [oracle_mod.splitmix64(1234567, r) for r in range(5)] == expect


def test_feistel_half_width_definition(oracle_mod):
    # B = max(2, 2*ceil(ceil(log2 m)/2)), h = B/2
    for m, h in [(2, 1), (3, 1), (4, 1), (5, 2), (16, 2), (17, 3), (64, 3), (65, 4),
                 (256, 4), (257, 5), (1024, 5), (1025, 6), (2048, 6), (4096, 6), (4097, 7)]:
        assert oracle_mod.half_bits(m) == h, m


@pytest.mark.parametrize("m", [2, 5, 17, 64, 257, 1025])
def test_feistel_is_bijection_on_domain(oracle_mod, m):
    dom = 1 << (2 * oracle_mod.half_bits(m))
    for seed in (0, 1, 2**63 + 5):
        img = [oracle_mod.feistel_enc(seed, m, x) for x in range(dom)]
        assert sorted(img) == list(range(dom))


@pytest.mark.parametrize("m", [3, 17, 300])
def test_feistel_dec_inverts_enc(oracle_mod, m):
    dom = 1 << (2 * oracle_mod.half_bits(m))
    for seed in (1, 77):
        for x in range(0, dom, max(1, dom // 257)):
            assert oracle_mod.feistel_dec(seed, m, oracle_mod.feistel_enc(seed, m, x)) == x


def test_visit_order_is_increasing_key_order(oracle_mod):
    # The keys of the visited constraints increase along the order.
    for m in (2, 9, 100, 1000):
        for seed in (4, 5):
            order = oracle_mod.perm_array(seed, m)
            keys = [oracle_mod.feistel_enc(seed, m, int(q)) for q in order]
            assert all(a < b for a, b in zip(keys, keys[1:]))


def test_perm_is_bijection_and_inverse(oracle_mod):
    sizes = list(range(0, 70)) + [255, 256, 257, 1000, 2047, 2048, 2049, 5000]
    for m in sizes:
        for seed in (3, 20190213 + m):
            p = oracle_mod.perm_array(seed, m)
            assert sorted(p.tolist()) == list(range(m))
            for k in range(0, m, max(1, m // 17)):
                assert oracle_mod.perm_inv(seed, m, int(p[k])) == k


def test_perm_not_identity_and_seed_dependent(oracle_mod):
    m = 256
    p1, p2 = oracle_mod.perm_array(11, m), oracle_mod.perm_array(12, m)
    assert (p1 != np.arange(m)).mean() > 0.9
    assert (p1 != p2).mean() > 0.9


@pytest.mark.parametrize("m", [16, 257])
def test_perm_first_position_uniform(oracle_mod, m):
    # Over many seeds, the constraint visited first is uniform on [0, m): chi-square.
    n = 200 * m
    counts = np.bincount([oracle_mod.perm_fwd(s, m, 0) for s in range(n)], minlength=m)
    exp = n / m
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # mean m-1, sd sqrt(2(m-1)); allow 5 sd
    assert abs(chi2 - (m - 1)) < 5 * math.sqrt(2 * (m - 1)), chi2


def test_perm_position_rank_uncorrelated(oracle_mod):
    m = 256
    rs = []
    for s in range(200):
        p = oracle_mod.perm_array(s, m)
        rs.append(np.corrcoef(np.arange(m), p)[0, 1])
    assert abs(np.mean(rs)) < 0.02 and np.std(rs) < 0.1


# ------------------------------------------------------------- hand-solved LPs
@pytest.mark.parametrize("case", lp_pins.load_hand_lps(), ids=lambda c: c["name"])
def test_hand_solved_golden(oracle_mod, case):
    # seeds 0 and 2 visit the two constraints of a two-constraint LP in both orders
    for seed in (0, 1, 2, 7):
        st, xy, _, _ = solve_one(oracle_mod, case["cons"], case["obj"], case["box"], seed)
        assert st == case["status"]
        if case["xyf"] is not None:
            x, y, f = case["xyf"]
            assert xy[0] == pytest.approx(x, abs=1e-9) and xy[1] == pytest.approx(y, abs=1e-9)
            c = case["obj"]
            assert c[0] * xy[0] + c[1] * xy[1] == pytest.approx(f, abs=1e-9)
        else:
            assert np.isnan(xy).all()


# ------------------------------------------------------------- brute force
def _tiny_lps(rng, n):
    for _ in range(n):
        m = int(rng.integers(0, 11))
        a = rng.normal(size=(m, 2)) * rng.uniform(0.2, 3.0, size=(m, 1))
        b = rng.normal(0.6, 1.0, size=m)
        half = float(rng.uniform(2.0, 40.0))
        box = (-half, half * rng.uniform(0.5, 1.5), -half * rng.uniform(0.5, 1.5), half)
        box = tuple(float(np.float32(v)) for v in box)
        c = rng.normal(size=2)
        yield (np.float32(a[:, 0]), np.float32(a[:, 1]), np.float32(b), np.float32(c), box)


def test_oracle_matches_brute_force(oracle_mod):
    rng = np.random.default_rng(1234)
    seen = np.zeros(3, int)
    for ax, ay, b, c, box in _tiny_lps(rng, 3000):
        cons = np.stack([ax, ay, b], axis=1)
        st, xy, _, _ = solve_one(oracle_mod, cons, c, box, seed=int(rng.integers(1 << 30)))
        bst, bxy, bf, _ = lp_pins.brute_force(ax.astype(float), ay.astype(float), b.astype(float),
                                               c.astype(float), box)
        seen[bst] += 1
        assert st == bst, (cons, c, box, xy, bxy)
        if bst != 1:
            f = float(c[0]) * xy[0] + float(c[1]) * xy[1]
            assert abs(f - bf) <= 1e-9 * max(1.0, abs(bf))
            assert abs(xy[0] - bxy[0]) <= 1e-7 * max(1.0, abs(bxy[0]))
            assert abs(xy[1] - bxy[1]) <= 1e-7 * max(1.0, abs(bxy[1]))
    assert seen.min() > 200, seen  # every outcome is exercised


# ------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [3, 4, 5, 8, 16, 33, 100])
def test_regular_ngon_closed_form(oracle_mod, n):
    rng = np.random.default_rng(n)
    for trial in range(6):
        r = float(rng.uniform(0.3, 2.0))
        c0 = rng.uniform(-1, 1, size=2)
        ang = 2 * math.pi * np.arange(n) / n
        nrm = np.stack([np.cos(ang), np.sin(ang)], axis=1)
        cons = np.concatenate([nrm, (r + nrm @ c0)[:, None]], axis=1)
        rng.shuffle(cons)
        j = int(rng.integers(n))
        # objective along a vertex direction: f = c.c0 + r / cos(pi/n)
        cv = np.array([math.cos(math.pi / n + 2 * math.pi * j / n), math.sin(math.pi / n + 2 * math.pi * j / n)])
        st, xy, _, _ = solve_one(oracle_mod, cons, cv, seed=trial)
        assert st == 0
        f32 = np.float32(cv).astype(float)
        expect = f32 @ c0 + r / math.cos(math.pi / n)
        assert f32 @ xy == pytest.approx(expect, abs=2e-6 * (1 + abs(expect)))
        # objective along a face normal: f = c.c0 + r (an edge of optima)
        cf = np.array([math.cos(2 * math.pi * j / n), math.sin(2 * math.pi * j / n)])
        st, xy, _, _ = solve_one(oracle_mod, cons, cf, seed=trial)
        assert st == 0
        f32 = np.float32(cf).astype(float)
        assert f32 @ xy == pytest.approx(f32 @ c0 + r, abs=2e-6 * (1 + r))


def test_empty_lp_is_box_corner(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(50):
        c = np.float32(rng.normal(size=2))
        st, xy, d, nv = solve_one(oracle_mod, np.zeros((0, 3)), c)
        assert st == 2 and nv == 0
        assert c.astype(float) @ xy == pytest.approx(abs(float(c[0])) * 1e3 + abs(float(c[1])) * 1e3)


def test_single_half_plane_is_box_bounded(oracle_mod):
    rng = np.random.default_rng(6)
    for _ in range(200):
        a = rng.normal(size=2)
        st, xy, d, _ = solve_one(oracle_mod, [[a[0], a[1], rng.normal()]], rng.normal(size=2))
        assert st == 2
        assert min(d[:2]) < 0


def test_antiparallel_pair_infeasible_and_strip(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(200):
        a = np.float32(rng.normal(size=2))
        st, xy, d, _ = solve_one(oracle_mod, [[a[0], a[1], -1], [-a[0], -a[1], -1]], rng.normal(size=2))
        assert st == 1 and np.isnan(xy).all()
        beta = float(rng.uniform(0.1, 3))
        st, xy, d, _ = solve_one(oracle_mod, [[a[0], a[1], beta], [-a[0], -a[1], beta]], rng.normal(size=2))
        assert st == 2  # c is never parallel to a for Gaussian draws


def test_bad_input_flagged(oracle_mod):
    st, xy, _, _ = solve_one(oracle_mod, [[1, 0, 1], [np.nan, 0, 1]], [1, 1])
    assert st == 3 and np.isnan(xy).all()
    st, _, _, _ = solve_one(oracle_mod, [[1, 0, np.inf]], [1, 1])
    assert st == 3
    st, _, _, _ = solve_one(oracle_mod, [[1, 0, 1]], [np.nan, 1])
    assert st == 3


# ----------------------------------------------------- certificates at scale
def _rows_of(batch, lp):
    s = int(batch["offsets"][lp])
    box = lp_pins.box_rows(batch["box"])

    def rows_of(i):
        if i < 0:
            return box[-1 - i]
        return (float(batch["ax"][s + i]), float(batch["ay"][s + i]), float(batch["b"][s + i]))
    return rows_of


@pytest.mark.parametrize("wl", ["plain_small", "plain_slice", "ragged_slice"])
def test_certificates_on_workloads(oracle_mod, wl):
    if wl == "plain_small":
        batch = workloads.plain_small()
    elif wl == "plain_slice":
        batch = workloads.plain_at_scale(n_lp=2048)
    else:
        batch = workloads.ragged(n_lp=2048)
    r = oracle_mod.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"],
                               batch["box"], seed=99, want_def=True)
    st, xy, dfn = r["status"], r["xy"], r["def"]
    assert ((st == 1) == batch["infeasible"]).all()
    for lp in range(len(st)):
        rows_of = _rows_of(batch, lp)
        s, e = batch["offsets"][lp], batch["offsets"][lp + 1]
        if st[lp] == 1:
            ids = [int(v) for v in dfn[lp] if v != oracle_mod.NONE_ID]
            lp_pins.farkas_certificate([rows_of(i) for i in ids])
            continue
        c = batch["obj"][lp].astype(float)
        lp_pins.kkt_certificate(rows_of, xy[lp], c, (int(dfn[lp][0]), int(dfn[lp][1])))
        A = np.stack([batch["ax"][s:e], batch["ay"][s:e]], 1).astype(float)
        slack = A @ xy[lp] - batch["b"][s:e]
        scale = max(1.0, np.abs(xy[lp]).max())
        assert slack.max(initial=-1) <= 1e-9 * scale * 4
        assert (st[lp] == 2) == (min(dfn[lp][:2]) < 0)


def test_order_independence(oracle_mod):
    batch = workloads.ragged(n_lp=1024)
    res = [oracle_mod.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"],
                                  batch["box"], seed=s) for s in (1, 2, 3)]
    f = [np.einsum("ij,ij->i", r["xy"], batch["obj"].astype(float)) for r in res]
    for k in (1, 2):
        assert (res[k]["status"] == res[0]["status"]).all()
        ok = res[0]["status"] != 1
        assert np.allclose(f[k][ok], f[0][ok], rtol=1e-12, atol=1e-12)


# ------------------------------------------------- random order does its job
def test_random_order_defeats_adversarial_input(oracle_mod):
    # Tangents to the unit circle stored in increasing angle over a quarter turn with
    # c = (0, 1): visiting them in stored order would violate at every step (the
    # optimum slides along the arc).  A random order needs O(log m) violations
    # in expectation (Sec. 2.1: expected O(m) total time).
    m = 512
    ang = np.linspace(0, math.pi / 2, m, endpoint=False)
    cons = np.stack([np.cos(ang), np.sin(ang), np.ones(m)], axis=1)
    nv = [solve_one(oracle_mod, cons, [0.0, 1.0], seed=s)[3] for s in range(20)]
    assert np.mean(nv) < 30, nv


def test_mean_violations_near_2_ln_m(oracle_mod):
    batch = workloads.disk_batch(np.full(4000, 256), seed=3)
    r = oracle_mod.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"],
                               batch["box"], seed=3, want_nviol=True)
    mean = r["nviol"].mean()
    assert 0.6 * 2 * math.log(256) < mean < 1.2 * 2 * math.log(256), mean


# ------------------------------------------------------ library cross-check
def test_against_scipy_highs(oracle_mod):
    sopt = pytest.importorskip("scipy.optimize")
    batch = workloads.ragged(n_lp=300, lo=8, hi=64)
    r = oracle_mod.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"],
                               batch["box"])
    xmin, xmax, ymin, ymax = batch["box"]
    for lp in range(300):
        s, e = batch["offsets"][lp], batch["offsets"][lp + 1]
        A = np.stack([batch["ax"][s:e], batch["ay"][s:e]], 1).astype(float)
        c = batch["obj"][lp].astype(float)
        res = sopt.linprog(-c, A_ub=A, b_ub=batch["b"][s:e].astype(float),
                           bounds=[(xmin, xmax), (ymin, ymax)], method="highs")
        if r["status"][lp] == 1:
            assert res.status == 2
        else:
            assert res.status == 0
            assert -res.fun == pytest.approx(c @ r["xy"][lp], rel=1e-7, abs=1e-7)


# ------------------------------------------------------ reading R3 (ties)
def duplicate_defining_constraint_batch(oracle, n_lp, seed):
    """LPs of the disk family, each with an exact copy of one constraint through its
    optimum appended: the constraint the oracle reports as the bound of the last 1-D
    LP (seed `seed`).  Returns the batch and, per LP, the indices (original, copy) of
    the duplicated pair.  Whenever the pair's line bounds a later 1-D LP, the two give
    equal sigma values, so the pair tests the tie rule (earliest position first)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(20), np.log(300), n_lp)).astype(np.int64)
    base = workloads.disk_batch(sizes, seed=seed, infeasible_frac=0.0)
    ref = oracle.solve_batch(base["ax"], base["ay"], base["b"], base["offsets"], base["obj"], base["box"],
                             seed=seed, want_def=True)
    cols = {k: [] for k in ("ax", "ay", "b")}
    pair, sz = [], []
    for l in range(n_lp):
        s, e = int(base["offsets"][l]), int(base["offsets"][l + 1])
        d = int(ref["def"][l][1])
        if ref["status"][l] != oracle.OPTIMAL or d < 0:
            d = 0  # any constraint: the LP then rarely exercises the rule
        for k in cols:
            v = base[k][s:e]
            cols[k].append(np.r_[v, v[d:d + 1]])
        pair.append((d, e - s))
        sz.append(e - s + 1)
    off = np.zeros(n_lp + 1, np.int64)
    np.cumsum(sz, out=off[1:])
    batch = {k: np.concatenate(v).astype(np.float32) for k, v in cols.items()}
    batch.update({"offsets": off, "obj": base["obj"], "box": base["box"]})
    return batch, np.asarray(pair, np.int64)

def test_duplicate_pair_reports_the_earlier_visited_copy(oracle_mod):
    # An exact copy of a constraint through the optimum: both copies give the same
    # sigma in every 1-D LP that they bound, and a later copy is never violated (the
    # optimum satisfies its twin).  So whichever of the two the oracle reports must be
    # the one visited first (reading R3), whatever the visit order.
    batch, pair = duplicate_defining_constraint_batch(oracle_mod, 600, seed=31)
    seed = 5
    ref = oracle_mod.solve_batch(batch["ax"], batch["ay"], batch["b"], batch["offsets"], batch["obj"], batch["box"],
                                 seed=seed, want_def=True)
    exercised = 0
    for l in range(len(pair)):
        d = ref["def"][l][:2]
        a, b = pair[l]
        hit = [x for x in d if x in (a, b)]
        if ref["status"][l] == oracle_mod.INFEASIBLE or not hit:
            continue
        m = int(batch["offsets"][l + 1] - batch["offsets"][l])
        pos = np.argsort(oracle_mod.perm_array(seed + l, m))  # visit position of each constraint
        assert len(hit) == 1
        assert pos[hit[0]] == min(pos[a], pos[b]), (l, d, a, b)
        exercised += 1
    assert exercised >= 400
