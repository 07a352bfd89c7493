/* seidel3_oracle.c -- FP64 CPU oracle for the batched 3-D LP solve.
 *
 * TEST INFRASTRUCTURE ONLY: called from tests/ (through oracle/__init__.py); the
 * product path never links or runs it.
 *
 * The paper describes Seidel's randomized incremental method for two dimensions
 * (Sec. 2.1) and names higher dimensions as the next step (Sec. 6).  This file
 * writes out the same method one dimension up, step by step:
 *   maximise c.x over x in R^3 subject to a_i.x <= b_i and the bounding box
 *   (the +-M constraints of Sec. 2.1, six planes in three dimensions);
 *   start at the box corner that maximises c;
 *   visit the constraints in the LP's random order; while the optimum satisfies the
 *   visited constraint keep it, otherwise the new optimum lies on that constraint's
 *   plane: solve the 2-D LP on the plane over the box and every earlier constraint,
 *   which is Seidel's 2-D method again, whose violations in turn solve 1-D LPs on
 *   lines (Eqs. 3 and 4).  An infeasible 2-D LP makes the 3-D LP infeasible.
 *
 * Readings (the paper is silent on them; R16-R21 of the project's readings):
 *   - box planes have positions -6..-1 in the order x<=xmax, -x<=-xmin, y<=ymax,
 *     -y<=-ymin, z<=zmax, -z<=-zmin, and ids -1..-6;
 *   - the visit order is the 2-D solver's (oracle_perm_array, seed + l);
 *   - the plane a.x = b is parameterised as p0 + s u + t w with p0 = a b / |a|^2,
 *     u = a x e_j (e_j the axis of the smallest |a_j|, the first on ties) and
 *     w = a x u;
 *   - the 2-D LP on the plane starts at the optimum over the six box planes alone,
 *     found by enumerating the intersections of pairs of them (the first pair in
 *     order wins ties);
 *   - violation tests use the 3-D point and the 2-D solver's relative tolerance:
 *     a.x - b > eps (|a_x x| + |a_y y| + |a_z z| + |b|);
 *   - 1-D LPs follow the 2-D solver's rules: strict comparisons (the earliest
 *     position wins ties, box first), den == 0 excludes the line iff num < 0, the
 *     left end is taken when the objective is perpendicular to the line.
 * The first-pair rule of the start, the orientation of the frame (w = a x u) and the
 * endpoint taken when the objective is orthogonal to the line decide which optimal
 * point a degenerate LP returns; hand-solved LPs pin each of them.  The axis e_j
 * itself changes no exact result (the direction of a line of the plane in R^3,
 * -(g.w) u + (g.u) w, does not depend on it), only rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define ORACLE3_OPTIMAL 0
#define ORACLE3_INFEASIBLE 1
#define ORACLE3_BOX_BOUNDED 2
#define ORACLE3_BAD_INPUT 3

void oracle_perm_array(uint64_t seed, int64_t m, int64_t* out);

typedef struct {
    const float *ax, *ay, *az, *b;
    const int64_t* order; /* order[k] = constraint visited at position k */
    double box[6];        /* xmin, xmax, ymin, ymax, zmin, zmax */
    double eps;
} lp3;

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double r[3]) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/* The constraint at visit position j (j < 0: box plane 6 + j) as g.x <= gb, with
 * its id (>= 0: the LP's own index; -1..-6: box planes). */
static void constraint_at(const lp3* L, int64_t j, double g[3], double* gb, int32_t* id) {
    if (j < 0) {
        int s = (int)(j + 6);
        g[0] = g[1] = g[2] = 0.0;
        int axis = s / 2;
        if (s % 2 == 0) { g[axis] = 1.0;  *gb = L->box[2 * axis + 1]; }
        else            { g[axis] = -1.0; *gb = -L->box[2 * axis]; }
        *id = -1 - s;
    } else {
        int64_t q = L->order[j];
        g[0] = (double)L->ax[q];
        g[1] = (double)L->ay[q];
        g[2] = (double)L->az[q];
        *gb = (double)L->b[q];
        *id = (int32_t)q;
    }
}

static int violates(const double g[3], double gb, const double x[3], double eps) {
    double s = dot3(g, x) - gb;
    double tol = eps * (fabs(g[0] * x[0]) + fabs(g[1] * x[1]) + fabs(g[2] * x[2]) + fabs(gb));
    return s > tol;
}

/* The plane h.x = hb as p0 + s u + t w (see the readings above). */
typedef struct {
    double p0[3], u[3], w[3];
} plane;

static void plane_frame(const double h[3], double hb, plane* F) {
    double n2 = dot3(h, h);
    for (int k = 0; k < 3; k++) F->p0[k] = h[k] * hb / n2;
    int j = 0;
    if (fabs(h[1]) < fabs(h[j])) j = 1;
    if (fabs(h[2]) < fabs(h[j])) j = 2;
    double e[3] = {0.0, 0.0, 0.0};
    e[j] = 1.0;
    cross3(h, e, F->u);
    cross3(h, F->u, F->w);
}

static void plane_point(const plane* F, double s, double t, double x[3]) {
    for (int k = 0; k < 3; k++) x[k] = F->p0[k] + s * F->u[k] + t * F->w[k];
}

/* Constraint g.x <= gb on the plane: gs s + gt t <= gr. */
static void project(const plane* F, const double g[3], double gb, double* gs, double* gt, double* gr) {
    *gs = dot3(g, F->u);
    *gt = dot3(g, F->w);
    *gr = gb - dot3(g, F->p0);
}

/* The 2-D LP on the plane h.x = hb over the box and positions 0..k-1.
 * On success writes the 3-D point x and the ids of the two constraints (besides h)
 * that define it; returns 1, or 0 when the 2-D LP is infeasible (def2 then holds
 * the constraint that could not be met and, where there is one, a second). */
static int solve_on_plane(const lp3* L, int64_t k, const double h[3], double hb, const double c[3], double x[3],
                          int32_t def2[2]) {
    const int32_t NONE = INT32_MIN;
    plane F;
    plane_frame(h, hb, &F);
    double cs = dot3(c, F.u), ct = dot3(c, F.w);

    /* start: the optimum over the six box planes alone */
    double bs[6], bt[6], br[6];
    int32_t bid[6];
    for (int i = 0; i < 6; i++) {
        double g[3], gb;
        constraint_at(L, i - 6, g, &gb, &bid[i]);
        project(&F, g, gb, &bs[i], &bt[i], &br[i]);
    }
    int found = 0;
    double best = 0.0, s = 0.0, t = 0.0;
    def2[0] = def2[1] = NONE;
    for (int i = 0; i < 6; i++) {
        for (int j = i + 1; j < 6; j++) {
            double det = bs[i] * bt[j] - bt[i] * bs[j];
            if (det == 0.0) continue;
            double ss = (br[i] * bt[j] - bt[i] * br[j]) / det;
            double tt = (bs[i] * br[j] - br[i] * bs[j]) / det;
            double xx[3];
            plane_point(&F, ss, tt, xx);
            int ok = 1;
            for (int f = 0; f < 6 && ok; f++) {
                double g[3], gb;
                int32_t gid;
                constraint_at(L, f - 6, g, &gb, &gid);
                if (f != i && f != j && violates(g, gb, xx, L->eps)) ok = 0;
            }
            if (!ok) continue;
            double val = cs * ss + ct * tt;
            if (!found || val > best) {
                found = 1;
                best = val;
                s = ss;
                t = tt;
                def2[0] = bid[i];
                def2[1] = bid[j];
            }
        }
    }
    if (!found) { /* the plane misses the box */
        def2[0] = def2[1] = NONE;
        return 0;
    }

    /* Seidel's 2-D method on the plane over positions 0..k-1 */
    for (int64_t j = 0; j < k; j++) {
        double g[3], gb;
        int32_t gid;
        constraint_at(L, j, g, &gb, &gid);
        double xx[3];
        plane_point(&F, s, t, xx);
        if (!violates(g, gb, xx, L->eps)) continue;
        double gs, gt, gr;
        project(&F, g, gb, &gs, &gt, &gr);
        double nn = gs * gs + gt * gt;
        if (nn == 0.0) { /* g's plane is parallel to h's and the whole plane violates it */
            def2[0] = gid;
            def2[1] = NONE;
            return 0;
        }
        /* the line gs s + gt t = gr on the plane: q0 + tau d */
        double q0s = gs * gr / nn, q0t = gt * gr / nn;
        double ds = -gt, dt = gs;
        double lo = -INFINITY, hi = INFINITY;
        int32_t id_lo = NONE, id_hi = NONE, par = NONE;
        for (int64_t f = -6; f < j; f++) {
            double fg[3], fb, fs, ft, fr;
            int32_t fid;
            constraint_at(L, f, fg, &fb, &fid);
            project(&F, fg, fb, &fs, &ft, &fr);
            double den = fs * ds + ft * dt;
            double num = fr - (fs * q0s + ft * q0t);
            if (den > 0.0) { /* bounds tau from above: Eq. 4 */
                double tau = num / den;
                if (tau < hi) { hi = tau; id_hi = fid; }
            } else if (den < 0.0) { /* from below: Eq. 3 */
                double tau = num / den;
                if (tau > lo) { lo = tau; id_lo = fid; }
            } else if (num < 0.0) {
                par = fid;
                break;
            }
        }
        if (par != NONE) {
            def2[0] = gid;
            def2[1] = par;
            return 0;
        }
        if (lo > hi) {
            def2[0] = gid;
            def2[1] = NONE;
            return 0;
        }
        double cd = cs * ds + ct * dt;
        double tau;
        int32_t e;
        if (cd > 0.0) { tau = hi; e = id_hi; }
        else          { tau = lo; e = id_lo; }
        s = q0s + tau * ds;
        t = q0t + tau * dt;
        def2[0] = gid;
        def2[1] = e;
    }
    plane_point(&F, s, t, x);
    return 1;
}

/* Solve one 3-D LP; box = {xmin, xmax, ymin, ymax, zmin, zmax}.  def[0..2]: the ids
 * of the three constraints through the returned vertex (OPTIMAL / BOX_BOUNDED), or of
 * the violated constraint and what made its plane infeasible (INFEASIBLE).
 * Returns the status. */
int32_t oracle_solve_lp3(const float* ax, const float* ay, const float* az, const float* b, int64_t m, const float* c_f,
                         const double box[6], uint64_t seed, double eps, double* xyz, int32_t* def,
                         int64_t* nviol_out) {
    const int32_t NONE = INT32_MIN;
    double c[3] = {(double)c_f[0], (double)c_f[1], (double)c_f[2]};
    def[0] = def[1] = def[2] = NONE;
    int bad = !isfinite(c[0]) || !isfinite(c[1]) || !isfinite(c[2]);
    for (int64_t i = 0; i < m && !bad; i++)
        if (!isfinite(ax[i]) || !isfinite(ay[i]) || !isfinite(az[i]) || !isfinite(b[i])) bad = 1;
    if (bad) {
        xyz[0] = xyz[1] = xyz[2] = NAN;
        if (nviol_out) *nviol_out = 0;
        return ORACLE3_BAD_INPUT;
    }
    int64_t* order = (int64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    oracle_perm_array(seed, m, order);
    lp3 L = {ax, ay, az, b, order, {box[0], box[1], box[2], box[3], box[4], box[5]}, eps};

    double x[3];
    for (int k = 0; k < 3; k++) {
        x[k] = (c[k] >= 0.0) ? box[2 * k + 1] : box[2 * k];
        def[k] = (c[k] >= 0.0) ? -1 - 2 * k : -2 - 2 * k;
    }
    int32_t status = -1;
    int64_t nviol = 0;
    for (int64_t k = 0; k < m; k++) {
        double h[3], hb;
        int32_t hid;
        constraint_at(&L, k, h, &hb, &hid);
        if (!violates(h, hb, x, eps)) continue;
        if (dot3(h, h) == 0.0) { /* 0.x <= hb < 0 */
            def[0] = hid; def[1] = def[2] = NONE;
            status = ORACLE3_INFEASIBLE;
            break;
        }
        int32_t d2[2];
        double xn[3];
        nviol++;
        if (!solve_on_plane(&L, k, h, hb, c, xn, d2)) {
            def[0] = hid; def[1] = d2[0]; def[2] = d2[1];
            status = ORACLE3_INFEASIBLE;
            break;
        }
        x[0] = xn[0]; x[1] = xn[1]; x[2] = xn[2];
        def[0] = hid; def[1] = d2[0]; def[2] = d2[1];
    }
    free(order);
    if (nviol_out) *nviol_out = nviol;
    if (status == ORACLE3_INFEASIBLE) {
        xyz[0] = xyz[1] = xyz[2] = NAN;
        return status;
    }
    xyz[0] = x[0]; xyz[1] = x[1]; xyz[2] = x[2];
    return (def[0] < 0 || def[1] < 0 || def[2] < 0) ? ORACLE3_BOX_BOUNDED : ORACLE3_OPTIMAL;
}

/* Solve LPs [lp_begin, lp_end) of a CSR batch: offsets[l]..offsets[l+1] is LP l's
 * slice of ax/ay/az/b, obj holds (cx, cy, cz) per LP, seed_l = seed + l.  out_xyz: 3
 * doubles per LP, out_status: 1 int, out_def: 3 ints or NULL, out_nviol: 1 int64 or
 * NULL. */
void oracle_solve_batch3(const float* ax, const float* ay, const float* az, const float* b, const int64_t* offsets,
                         int64_t lp_begin, int64_t lp_end, const float* obj, const double* box, uint64_t seed,
                         double eps, double* out_xyz, int32_t* out_status, int32_t* out_def, int64_t* out_nviol) {
    for (int64_t l = lp_begin; l < lp_end; l++) {
        int64_t o = offsets[l];
        int64_t m = offsets[l + 1] - o;
        int32_t def[3];
        int64_t nv = 0;
        out_status[l] = oracle_solve_lp3(ax + o, ay + o, az + o, b + o, m, obj + 3 * l, box, seed + (uint64_t)l, eps,
                                         out_xyz + 3 * l, def, &nv);
        if (out_def) { out_def[3 * l] = def[0]; out_def[3 * l + 1] = def[1]; out_def[3 * l + 2] = def[2]; }
        if (out_nviol) out_nviol[l] = nv;
    }
}
