"""Planted mistakes in the oracles fail their pins.

Each case copies the oracle's C sources, plants one plausible mistake in one of them
(a flipped comparison or sign, a dropped constraint, a wrong corner, a wrong
coefficient), builds the copy, swaps it in for the oracle's library and runs a few
of the pin tests against it: at least one must fail.  An unplanted copy passes the
same pins, so the failures come from the mistakes.  Every planted mistake keeps all
memory accesses in bounds.  CPU only."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import pytest

import lp_pins
import oracle
import test_oracle3_pins as pins3
import test_oracle_pins as pins2
import test_oracleN_pins as pinsN

SRC_DIR = os.path.dirname(oracle.__file__)
SOURCES = ("seidel_oracle.c", "seidel3_oracle.c", "seidelN_oracle.c")

DETECT_2D = [
    lambda: pins2.test_oracle_matches_brute_force(oracle),
    lambda: pins2.test_regular_ngon_closed_form(oracle, 8),
    lambda: [pins2.test_hand_solved_golden(oracle, case) for case in lp_pins.load_hand_lps()],
    lambda: pins2.test_antiparallel_pair_infeasible_and_strip(oracle),
    lambda: pins2.test_duplicate_pair_reports_the_earlier_visited_copy(oracle),
]
DETECT_3D = [pins3.test_brute_force_on_tiny_lps, pins3.test_cube_and_box_closed_forms,
             pins3.test_octahedron_closed_form, pins3.test_every_hand_solved_degenerate_golden]
DETECT_ND = [
    lambda: pinsN.test_brute_force_on_tiny_lps(4, 500),
    lambda: pinsN.test_hypercube_cross_polytope_and_simplex_closed_forms(4),
    lambda: pinsN.test_kkt_certificates_on_a_generated_batch(4),
    pinsN.test_every_hand_solved_degenerate_golden,
]

# (name, file, text, replacement, detectors)
MUTATIONS = [
    ("2d_objective_end", "seidel_oracle.c", "if (cu > 0.0) { t = u_right; e = id_right; }",
     "if (cu < 0.0) { t = u_right; e = id_right; }", DETECT_2D),
    ("2d_right_bound_max", "seidel_oracle.c", "if (t < u_right) { u_right = t; id_right = gid; }",
     "if (t > u_right) { u_right = t; id_right = gid; }", DETECT_2D),
    ("2d_last_earlier_dropped", "seidel_oracle.c", "for (int64_t j = -4; j < i; j++) {",
     "for (int64_t j = -4; j < i - 1; j++) {", DETECT_2D),
    ("2d_wrong_start_corner", "seidel_oracle.c", "double x0 = (cx >= 0.0) ? box[1] : box[0];",
     "double x0 = (cx >= 0.0) ? box[0] : box[1];", DETECT_2D),
    ("2d_line_direction", "seidel_oracle.c", "double ux = -hy, uy = hx;", "double ux = hy, uy = hx;", DETECT_2D),
    ("2d_endpoint_reading_r2", "seidel_oracle.c", "if (cu > 0.0) { t = u_right; e = id_right; }",
     "if (cu >= 0.0) { t = u_right; e = id_right; }", DETECT_2D),
    ("2d_tie_reading_r3_left", "seidel_oracle.c", "if (t > u_left) { u_left = t; id_left = gid; }",
     "if (t >= u_left) { u_left = t; id_left = gid; }", DETECT_2D),
    ("2d_tie_reading_r3_right", "seidel_oracle.c", "if (t < u_right) { u_right = t; id_right = gid; }",
     "if (t <= u_right) { u_right = t; id_right = gid; }", DETECT_2D),
    ("2d_parallel_rule", "seidel_oracle.c", "} else if (num < 0.0) {  /* parallel and excluding the line */",
     "} else if (num > 0.0) {  /* parallel and excluding the line */", DETECT_2D),
    ("3d_objective_end", "seidel3_oracle.c", "if (cd > 0.0) { tau = hi; e = id_hi; }",
     "if (cd < 0.0) { tau = hi; e = id_hi; }", DETECT_3D),
    ("3d_start_minimum", "seidel3_oracle.c", "if (!found || val > best) {", "if (!found || val < best) {", DETECT_3D),
    ("3d_last_earlier_dropped", "seidel3_oracle.c", "for (int64_t f = -6; f < j; f++) {",
     "for (int64_t f = -6; f < j - 1; f++) {", DETECT_3D),
    ("3d_wrong_start_corner", "seidel3_oracle.c", "x[k] = (c[k] >= 0.0) ? box[2 * k + 1] : box[2 * k];",
     "x[k] = (c[k] >= 0.0) ? box[2 * k] : box[2 * k + 1];", DETECT_3D),
    ("3d_start_tie_last_pair_r18", "seidel3_oracle.c", "if (!found || val > best) {",
     "if (!found || val >= best) {", DETECT_3D),
    ("3d_frame_mirrored_r17", "seidel3_oracle.c", "cross3(h, F->u, F->w);", "cross3(F->u, h, F->w);", DETECT_3D),
    ("3d_endpoint_reading_r2", "seidel3_oracle.c", "if (cd > 0.0) { tau = hi; e = id_hi; }",
     "if (cd >= 0.0) { tau = hi; e = id_hi; }", DETECT_3D),
    ("nd_start_tie_last_subset_r24", "seidelN_oracle.c", "if (!found || val > best) {",
     "if (!found || val >= best) {", DETECT_ND),
    ("nd_pivot_last_on_ties_r23", "seidelN_oracle.c", "if (fabs(A[i]) > fabs(A[J])) J = i;",
     "if (fabs(A[i]) >= fabs(A[J])) J = i;", DETECT_ND),
    ("nd_endpoint_reading_r2", "seidelN_oracle.c", "double s[DMAX] = {ce > 0.0 ? hi : lo};",
     "double s[DMAX] = {ce >= 0.0 ? hi : lo};", DETECT_ND),
    ("nd_objective_end", "seidelN_oracle.c", "double s[DMAX] = {ce > 0.0 ? hi : lo};",
     "double s[DMAX] = {ce < 0.0 ? hi : lo};", DETECT_ND),
    ("nd_frame_point_sign", "seidelN_oracle.c", "T.p[t] = S->p[t] + (r / A[J]) * S->E[J][t];",
     "T.p[t] = S->p[t] - (r / A[J]) * S->E[J][t];", DETECT_ND),
    ("nd_frame_basis_sign", "seidelN_oracle.c", "T.E[n][t] = S->E[i][t] - (A[i] / A[J]) * S->E[J][t];",
     "T.E[n][t] = S->E[i][t] + (A[i] / A[J]) * S->E[J][t];", DETECT_ND),
    ("nd_start_minimum", "seidelN_oracle.c", "if (!found || val > best) {", "if (!found || val < best) {",
     DETECT_ND),
    ("nd_last_earlier_dropped", "seidelN_oracle.c", "if (!solve_sub(L, &T, j, x, dn))",
     "if (!solve_sub(L, &T, j > 0 ? j - 1 : 0, x, dn))", DETECT_ND),
    ("nd_box_side_bound", "seidelN_oracle.c", "if (s % 2 == 0) { g[axis] = 1.0;  *gb = L->box[2 * axis + 1]; }",
     "if (s % 2 == 0) { g[axis] = 1.0;  *gb = L->box[2 * axis]; }", DETECT_ND),
    ("nd_wrong_coefficient", "seidelN_oracle.c", "for (int t = 0; t < L->d; t++) g[t] = (double)L->a[q * L->d + t];",
     "for (int t = 0; t < L->d; t++) g[t] = (double)L->a[q * L->d + (t + 1) % L->d];", DETECT_ND),
]


def build_copy(tmp_path, mutation=None):
    """Build a copy of the oracle library, with `mutation` (file, text, replacement)
    planted, and bind it like the oracle's own."""
    for name in SOURCES:
        shutil.copy(os.path.join(SRC_DIR, name), tmp_path / name)
    if mutation is not None:
        fname, text, replacement = mutation
        src = (tmp_path / fname).read_text()
        assert src.count(text) == 1, f"the text to mutate must occur once in {fname}: {text}"
        (tmp_path / fname).write_text(src.replace(text, replacement))
    lib_path = tmp_path / "liboracle_copy.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(lib_path),
                           *[str(tmp_path / n) for n in SOURCES], "-lm"])
    return oracle._bind(ctypes.CDLL(str(lib_path)))


def failures(detectors):
    n = 0
    for detect in detectors:
        try:
            detect()
        except AssertionError:
            n += 1
    return n


def test_the_unplanted_copy_passes_every_detector(tmp_path, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", build_copy(tmp_path))
    assert failures(DETECT_2D + DETECT_3D + DETECT_ND) == 0


@pytest.mark.parametrize("name,fname,text,replacement,detectors", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(name, fname, text, replacement, detectors, tmp_path, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", build_copy(tmp_path, (fname, text, replacement)))
    assert failures(detectors) >= 1, f"no pin caught the planted mistake {name}"
