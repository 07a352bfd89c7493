/* seidelN_oracle.c -- FP64 CPU oracle for batched LPs in d = 1..5 dimensions.
 *
 * TEST INFRASTRUCTURE ONLY: called from tests/ (through oracle/__init__.py); the
 * product path never links or runs it.
 *
 * Seidel's randomized incremental method (Sec. 2.1 gives it in two dimensions, Sec. 6
 * names higher ones) in any dimension d, written as a recursion over affine
 * subspaces of R^d:
 *   maximise c.x subject to a_i.x <= b_i and the bounding box (2d planes, the +-M
 *   constraints of Sec. 2.1);
 *   a subspace of dimension k is x = p + sum_i s_i E_i (E_0..E_{k-1} vectors of R^d);
 *   on it, visit the constraints in the LP's random order from the best vertex of the
 *   box; keep the current point while it satisfies the visited constraint, otherwise
 *   solve the LP of dimension k - 1 on that constraint's hyperplane over the box and
 *   every earlier constraint, and an infeasible lower-dimensional LP makes the LP
 *   infeasible;
 *   dimension 1 is the 1-D LP of Eqs. 3 and 4 over the box and the earlier constraints.
 *
 * Readings (R22-R25 of the project's readings):
 *   - box planes have positions -2d..-1 in the order x_0 <= max_0, -x_0 <= -min_0,
 *     x_1 <= max_1, ... and ids -1..-2d;
 *   - the visit order is the 2-D solver's (oracle_perm_array, seed + l);
 *   - a subspace of dimension k >= 2 (the whole space included) starts at the best
 *     intersection of k box planes that satisfies the other box planes: all k-subsets
 *     in lexicographic order, the first wins ties, a subset whose planes are not
 *     independent in the subspace is skipped (in R^d this is the box corner that
 *     maximises c, the max side where c_j = 0);
 *   - the hyperplane A.s = r of a subspace (A_i = a.E_i, r = b - a.p) is the subspace
 *     p' = p + (r / A_J) E_J, E'_i = E_i - (A_i / A_J) E_J (i != J), with J the index
 *     of the largest |A_J| (the first on ties); A = 0 means the constraint's normal is
 *     orthogonal to the subspace, and a violated one then excludes all of it;
 *   - violation tests use the point in R^d with the 2-D solver's relative tolerance:
 *     a.x - b > eps (sum_j |a_j x_j| + |b|);
 *   - 1-D LPs on p + s E_0: strict comparisons (the earliest position wins ties, box
 *     first), a constraint with A = 0 excludes the line iff r < 0; the end at larger s
 *     is taken iff c.E_0 > 0; infeasible iff the left end exceeds the right end.
 * The tie rules of the start (the first k-subset among equally good box vertices) and
 * of the pivot (the first J among equal |A_J|) and the endpoint rule decide which
 * optimal point a degenerate LP returns; hand-solved LPs pin each of them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define ORACLEN_OPTIMAL 0
#define ORACLEN_INFEASIBLE 1
#define ORACLEN_BOX_BOUNDED 2
#define ORACLEN_BAD_INPUT 3
#define DMAX 5
#define NONE_ID INT32_MIN

void oracle_perm_array(uint64_t seed, int64_t m, int64_t* out);

typedef struct {
    int d;
    const float* a;       /* row-major [m][d] */
    const float* b;
    const int64_t* order; /* visit position -> constraint index */
    const double* box;    /* min_0, max_0, min_1, max_1, ... */
    const double* c;
    double eps;
    int64_t nviol;        /* violations in the whole space */
} lpn;

/* A subspace of dimension k: x = p + sum_i s_i E[i]. */
typedef struct {
    int k;
    double p[DMAX];
    double E[DMAX][DMAX];
} subspace;

/* The constraint at visit position j (j < 0: box plane 2d + j) as g.x <= gb, and its id. */
static void cons_at(const lpn* L, int64_t j, double g[DMAX], double* gb, int32_t* id) {
    for (int t = 0; t < L->d; t++) g[t] = 0.0;
    if (j < 0) {
        int s = (int)(j + 2 * L->d);
        int axis = s / 2;
        if (s % 2 == 0) { g[axis] = 1.0;  *gb = L->box[2 * axis + 1]; }
        else            { g[axis] = -1.0; *gb = -L->box[2 * axis]; }
        *id = -1 - s;
    } else {
        int64_t q = L->order[j];
        for (int t = 0; t < L->d; t++) g[t] = (double)L->a[q * L->d + t];
        *gb = (double)L->b[q];
        *id = (int32_t)q;
    }
}

static int violates(const lpn* L, const double g[DMAX], double gb, const double x[DMAX]) {
    double s = -gb, tol = fabs(gb);
    for (int t = 0; t < L->d; t++) {
        s += g[t] * x[t];
        tol += fabs(g[t] * x[t]);
    }
    return s > L->eps * tol;
}

static void sub_point(const lpn* L, const subspace* S, const double s[DMAX], double x[DMAX]) {
    for (int t = 0; t < L->d; t++) {
        x[t] = S->p[t];
        for (int i = 0; i < S->k; i++) x[t] += s[i] * S->E[i][t];
    }
}

/* g.x <= gb restricted to S: A.s <= r. */
static void sub_cons(const lpn* L, const subspace* S, const double g[DMAX], double gb, double A[DMAX], double* r) {
    double gp = 0.0;
    for (int t = 0; t < L->d; t++) gp += g[t] * S->p[t];
    *r = gb - gp;
    for (int i = 0; i < S->k; i++) {
        double v = 0.0;
        for (int t = 0; t < L->d; t++) v += g[t] * S->E[i][t];
        A[i] = v;
    }
}

/* M y = r (k x k) by Gaussian elimination with partial pivoting; 0 if singular. */
static int solve_k(int k, double M[DMAX][DMAX], double r[DMAX], double y[DMAX]) {
    for (int col = 0; col < k; col++) {
        int piv = col;
        for (int i = col + 1; i < k; i++)
            if (fabs(M[i][col]) > fabs(M[piv][col])) piv = i;
        if (M[piv][col] == 0.0) return 0;
        if (piv != col) {
            for (int j = 0; j < k; j++) { double t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t; }
            double t = r[col]; r[col] = r[piv]; r[piv] = t;
        }
        for (int i = col + 1; i < k; i++) {
            double f = M[i][col] / M[col][col];
            for (int j = col; j < k; j++) M[i][j] -= f * M[col][j];
            r[i] -= f * r[col];
        }
    }
    for (int i = k - 1; i >= 0; i--) {
        double v = r[i];
        for (int j = i + 1; j < k; j++) v -= M[i][j] * y[j];
        y[i] = v / M[i][i];
    }
    return 1;
}

/* The best vertex of the box inside S (dimension k >= 2): x and the ids of its k box
 * planes; 0 if S misses the box. */
static int box_vertex(const lpn* L, const subspace* S, double x[DMAX], int32_t def[DMAX]) {
    const int k = S->k, nb = 2 * L->d;
    int idx[DMAX], found = 0;
    double best = 0.0;
    for (int i = 0; i < k; i++) idx[i] = i;
    for (;;) {
        double M[DMAX][DMAX], r[DMAX], y[DMAX], A[DMAX], rr, g[DMAX], gb;
        int32_t ids[DMAX], gid;
        for (int i = 0; i < k; i++) {
            cons_at(L, idx[i] - nb, g, &gb, &ids[i]);
            sub_cons(L, S, g, gb, A, &rr);
            for (int j = 0; j < k; j++) M[i][j] = A[j];
            r[i] = rr;
        }
        if (solve_k(k, M, r, y)) {
            double xx[DMAX];
            sub_point(L, S, y, xx);
            int ok = 1;
            for (int f = 0, i = 0; f < nb && ok; f++) {
                if (i < k && idx[i] == f) { i++; continue; }
                cons_at(L, f - nb, g, &gb, &gid);
                if (violates(L, g, gb, xx)) ok = 0;
            }
            if (ok) {
                double val = 0.0;
                for (int t = 0; t < L->d; t++) val += L->c[t] * xx[t];
                if (!found || val > best) {
                    found = 1;
                    best = val;
                    for (int t = 0; t < L->d; t++) x[t] = xx[t];
                    for (int i = 0; i < k; i++) def[i] = ids[i];
                }
            }
        }
        int i = k - 1; /* next k-subset of 0..nb-1 in lexicographic order */
        while (i >= 0 && idx[i] == nb - k + i) i--;
        if (i < 0) break;
        idx[i]++;
        for (int j = i + 1; j < k; j++) idx[j] = idx[j - 1] + 1;
    }
    return found;
}

/* The LP on S over the box and visit positions 0..limit-1: the point x in R^d and the
 * ids of the k constraints that define it (def[0] = the constraint that made it
 * infeasible on failure).  Returns 1, or 0 when infeasible. */
static int solve_sub(lpn* L, const subspace* S, int64_t limit, double x[DMAX], int32_t def[DMAX]) {
    const int d = L->d, k = S->k;
    double g[DMAX], gb, A[DMAX], r;
    int32_t gid;
    if (k == 1) { /* Eqs. 3 and 4 on the line p + s E_0 */
        double lo = -INFINITY, hi = INFINITY, ce = 0.0;
        int32_t id_lo = NONE_ID, id_hi = NONE_ID;
        for (int64_t f = -2 * d; f < limit; f++) {
            cons_at(L, f, g, &gb, &gid);
            sub_cons(L, S, g, gb, A, &r);
            if (A[0] > 0.0) { double t = r / A[0]; if (t < hi) { hi = t; id_hi = gid; } }
            else if (A[0] < 0.0) { double t = r / A[0]; if (t > lo) { lo = t; id_lo = gid; } }
            else if (r < 0.0) { def[0] = gid; return 0; }
        }
        if (lo > hi) { def[0] = NONE_ID; return 0; }
        for (int t = 0; t < d; t++) ce += L->c[t] * S->E[0][t];
        double s[DMAX] = {ce > 0.0 ? hi : lo};
        def[0] = ce > 0.0 ? id_hi : id_lo;
        sub_point(L, S, s, x);
        return 1;
    }
    if (!box_vertex(L, S, x, def)) { def[0] = NONE_ID; return 0; }
    for (int64_t j = 0; j < limit; j++) {
        cons_at(L, j, g, &gb, &gid);
        if (!violates(L, g, gb, x)) continue;
        if (k == d) L->nviol++;
        sub_cons(L, S, g, gb, A, &r);
        int J = 0;
        for (int i = 1; i < k; i++)
            if (fabs(A[i]) > fabs(A[J])) J = i;
        if (A[J] == 0.0) { def[0] = gid; return 0; }
        subspace T; /* the hyperplane A.s = r inside S */
        T.k = k - 1;
        for (int t = 0; t < d; t++) T.p[t] = S->p[t] + (r / A[J]) * S->E[J][t];
        for (int i = 0, n = 0; i < k; i++) {
            if (i == J) continue;
            for (int t = 0; t < d; t++) T.E[n][t] = S->E[i][t] - (A[i] / A[J]) * S->E[J][t];
            n++;
        }
        int32_t dn[DMAX];
        if (!solve_sub(L, &T, j, x, dn)) { def[0] = gid; return 0; }
        def[0] = gid;
        for (int i = 0; i < k - 1; i++) def[i + 1] = dn[i];
    }
    return 1;
}

/* One LP in d dimensions (1 <= d <= 5): a row-major [m][d], b [m], c [d], box
 * {min_0, max_0, ..., min_{d-1}, max_{d-1}}.  Writes x [d], def [d] (the ids of the d
 * constraints through x; box planes are -1..-2d) and the number of violations in the
 * whole space; returns the status. */
int32_t oracle_solve_lpN(int d, const float* a, const float* b, int64_t m, const float* c_f, const double* box,
                         uint64_t seed, double eps, double* x_out, int32_t* def, int64_t* nviol_out) {
    int bad = d < 1 || d > DMAX;
    for (int t = 0; t < d && !bad; t++) bad |= !isfinite(c_f[t]);
    for (int64_t i = 0; i < m * d && !bad; i++) bad |= !isfinite(a[i]);
    for (int64_t i = 0; i < m && !bad; i++) bad |= !isfinite(b[i]);
    for (int t = 0; t < d && t < DMAX; t++) def[t] = NONE_ID;
    if (nviol_out) *nviol_out = 0;
    if (bad) {
        for (int t = 0; t < d && t < DMAX; t++) x_out[t] = NAN;
        return ORACLEN_BAD_INPUT;
    }
    int64_t* order = (int64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    oracle_perm_array(seed, m, order);
    double c[DMAX], x[DMAX];
    for (int t = 0; t < d; t++) c[t] = (double)c_f[t];
    lpn L = {d, a, b, order, box, c, eps, 0};
    subspace S; /* the whole space */
    S.k = d;
    for (int t = 0; t < d; t++) {
        S.p[t] = 0.0;
        for (int u = 0; u < d; u++) S.E[t][u] = (t == u) ? 1.0 : 0.0;
    }
    int feasible = solve_sub(&L, &S, m, x, def);
    free(order);
    if (nviol_out) *nviol_out = L.nviol;
    if (!feasible) {
        for (int t = 1; t < d; t++) def[t] = NONE_ID;
        for (int t = 0; t < d; t++) x_out[t] = NAN;
        return ORACLEN_INFEASIBLE;
    }
    int box_def = 0;
    for (int t = 0; t < d; t++) {
        x_out[t] = x[t];
        box_def |= def[t] < 0;
    }
    return box_def ? ORACLEN_BOX_BOUNDED : ORACLEN_OPTIMAL;
}

/* LPs [lp_begin, lp_end) of a CSR batch in d dimensions: a row-major
 * [n_constraints][d], LP l owns rows offsets[l]..offsets[l+1]-1, obj [n_lp][d], box 2d
 * values, seed_l = seed + l.  out_x: d doubles per LP; out_def: d ids per LP or NULL;
 * out_nviol: violations in the whole space or NULL. */
void oracle_solve_batchN(int d, const float* a, const float* b, const int64_t* offsets, int64_t lp_begin,
                         int64_t lp_end, const float* obj, const double* box, uint64_t seed, double eps,
                         double* out_x, int32_t* out_status, int32_t* out_def, int64_t* out_nviol) {
    for (int64_t l = lp_begin; l < lp_end; l++) {
        int64_t o = offsets[l];
        int64_t m = offsets[l + 1] - o;
        int32_t def[DMAX];
        int64_t nv = 0;
        out_status[l] = oracle_solve_lpN(d, a + o * d, b + o, m, obj + l * d, box, seed + (uint64_t)l, eps,
                                         out_x + l * d, def, &nv);
        if (out_def)
            for (int t = 0; t < d; t++) out_def[l * d + t] = def[t];
        if (out_nviol) out_nviol[l] = nv;
    }
}
