/*
 * seidel_oracle.c -- plain, serial, FP64 CPU oracle for the batched 2-D LP solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file; only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg do.  It shares no code, header or constant table with the CUDA library.
 *
 * What it computes (Charlton, Maddock & Richmond, "Two-Dimensional Batch Linear
 * Programming on the GPU", arXiv 1902.04995):
 *   - the LP  max c^T x  s.t.  A x <= b  in n = 2 dimensions (Sec. 2.1, Eq. 1, Eq. 2);
 *   - made bounded by the four box constraints x <= M, x >= -M per dimension
 *     (Sec. 2.1, the bounding-constraint trick);
 *   - solved by Seidel's randomized incremental method (Sec. 2.1): constraints are
 *     visited in a random order; a satisfied constraint leaves the optimum alone, a
 *     violated one moves the optimum onto its line, found by a 1-D LP over all
 *     earlier constraints (Eq. 3: u_left = max over left-bounded sigma(h,l),
 *     Eq. 4: u_right = min over right-bounded sigma(h,l); infeasible when the
 *     interval is empty; otherwise the endpoint favoured by the objective).
 *
 * Readings where the paper is silent or ambiguous (R1-R15 of the project's readings):
 *   - Eq. 3/4 infeasibility: strict u_left > u_right (a single point is feasible).
 *   - objective orthogonal to the line (c.u == 0): take u_left.
 *   - ties in sigma: the earliest visit position wins (box sides first, at
 *     positions -4..-1 in the order x<=xmax, x>=xmin, y<=ymax, y>=ymin).
 *   - a constraint parallel to the line (den == 0 exactly) is ignored when its
 *     offset admits the line and makes the LP infeasible otherwise (Sec. 2.1).
 *   - the 1-D LP runs over the box plus every constraint visited strictly before
 *     the violated one.
 *   - a zero normal (0,0) is infeasible when b < 0 and never violated otherwise.
 *   - violation test: a.x - b > eps * (|a_x x| + |a_y y| + |b|).
 *   - the random visit order (Sec. 2.1 asks for a random order, no generator is
 *     named): the constraints of LP l are visited in increasing order of their key
 *     E(q), where E is a 4-round balanced Feistel network on B = max(2,
 *     2*ceil(ceil(log2 m)/2)) bits (a bijection of [0, 2^B), so keys are distinct).
 *     Round key r is the low 32 bits of output r+1 of SplitMix64 (Steele, Lea &
 *     Flood, OOPSLA 2014) seeded with seed_l = seed + l.  Round function
 *     F(R, K) = top h bits of ((R xor K) * 0x9E3779B1 mod 2^32), h = B/2.
 *   - status BOX_BOUNDED: one of the two constraints defining the returned vertex
 *     is a box side.  Inputs with NaN/Inf give BAD_INPUT.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so x86 and
 * aarch64 hosts give bit-identical results).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OPTIMAL 0
#define ORACLE_INFEASIBLE 1
#define ORACLE_BOX_BOUNDED 2
#define ORACLE_BAD_INPUT 3

/* ---------------------------------------------------------------- SplitMix64 */
/* Output number (r + 1) of SplitMix64 seeded with `seed`: the state advances by the
 * golden gamma and the result is the published mix of the new state. */
uint64_t oracle_splitmix64(uint64_t seed, uint32_t r) {
    uint64_t z = seed + (uint64_t)(r + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ---------------------------------------------------------- visit order pi */
typedef struct {
    uint32_t key[4];
    uint32_t h;     /* bits per Feistel half; B = 2h */
    uint64_t m;
} oracle_perm;

static void perm_init(oracle_perm* P, uint64_t seed, uint64_t m) {
    P->m = m;
    uint32_t bits = 0; /* ceil(log2 m) */
    while (bits < 64 && ((uint64_t)1 << bits) < m) bits++;
    uint32_t h = (bits + 1) / 2;
    if (h < 1) h = 1;
    P->h = h;
    for (uint32_t r = 0; r < 4; r++) P->key[r] = (uint32_t)oracle_splitmix64(seed, r);
}

static uint32_t feistel_round_fn(uint32_t R, uint32_t K, uint32_t h) {
    uint32_t x = (R ^ K) * 0x9E3779B1u;
    return x >> (32u - h);
}

/* One encryption over the 2h-bit domain: (L, R) -> (R, L ^ F(R)), four rounds. */
static uint64_t feistel_enc(const oracle_perm* P, uint64_t x) {
    uint32_t h = P->h;
    uint32_t mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
    uint32_t L = (uint32_t)(x >> h) & mask;
    uint32_t R = (uint32_t)x & mask;
    for (int r = 0; r < 4; r++) {
        uint32_t nl = R;
        uint32_t nr = L ^ feistel_round_fn(R, P->key[r], h);
        L = nl;
        R = nr;
    }
    return ((uint64_t)L << h) | R;
}

static uint64_t feistel_dec(const oracle_perm* P, uint64_t x) {
    uint32_t h = P->h;
    uint32_t mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
    uint32_t L = (uint32_t)(x >> h) & mask;
    uint32_t R = (uint32_t)x & mask;
    for (int r = 3; r >= 0; r--) {
        uint32_t pl = R ^ feistel_round_fn(L, P->key[r], h);
        uint32_t pr = L;
        L = pl;
        R = pr;
    }
    return ((uint64_t)L << h) | R;
}

/* Visit order: sort the constraints by key.  order[k] = pi(k). */
typedef struct {
    uint64_t key;
    int64_t q;
} keyed;

static int keyed_cmp(const void* a, const void* b) {
    const keyed* x = (const keyed*)a;
    const keyed* y = (const keyed*)b;
    return (x->key > y->key) - (x->key < y->key);
}

static void visit_order(const oracle_perm* P, int64_t m, int64_t* order) {
    if (m <= 0) return;
    keyed* kq = (keyed*)malloc((size_t)m * sizeof(keyed));
    for (int64_t q = 0; q < m; q++) {
        kq[q].key = feistel_enc(P, (uint64_t)q);
        kq[q].q = q;
    }
    qsort(kq, (size_t)m, sizeof(keyed), keyed_cmp);
    for (int64_t k = 0; k < m; k++) order[k] = kq[k].q;
    free(kq);
}

int64_t oracle_perm_fwd(uint64_t seed, int64_t m, int64_t k) {
    oracle_perm P;
    perm_init(&P, seed, (uint64_t)m);
    int64_t* order = (int64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    visit_order(&P, m, order);
    int64_t r = order[k];
    free(order);
    return r;
}

/* Position of constraint q: the number of constraints with a smaller key. */
int64_t oracle_perm_inv(uint64_t seed, int64_t m, int64_t q) {
    oracle_perm P;
    perm_init(&P, seed, (uint64_t)m);
    uint64_t kq = feistel_enc(&P, (uint64_t)q);
    int64_t rank = 0;
    for (int64_t i = 0; i < m; i++)
        if (feistel_enc(&P, (uint64_t)i) < kq) rank++;
    return rank;
}

/* Raw Feistel encryption on the 2h-bit domain (exposed for bijectivity tests). */
int64_t oracle_feistel_enc(uint64_t seed, int64_t m, int64_t x) {
    oracle_perm P;
    perm_init(&P, seed, (uint64_t)m);
    return (int64_t)feistel_enc(&P, (uint64_t)x);
}

/* Inverse Feistel (exposed for tests). */
int64_t oracle_feistel_dec(uint64_t seed, int64_t m, int64_t x) {
    oracle_perm P;
    perm_init(&P, seed, (uint64_t)m);
    return (int64_t)feistel_dec(&P, (uint64_t)x);
}

int32_t oracle_feistel_half_bits(int64_t m) {
    oracle_perm P;
    perm_init(&P, 0, (uint64_t)m);
    return (int32_t)P.h;
}

void oracle_perm_array(uint64_t seed, int64_t m, int64_t* out) {
    oracle_perm P;
    perm_init(&P, seed, (uint64_t)m);
    visit_order(&P, m, out);
}

/* ------------------------------------------------------------- one LP solve */
/* Box side s (0..3) as a constraint g.x <= gb:
 *   0: ( 1, 0).x <= xmax   1: (-1, 0).x <= -xmin   2: (0, 1).x <= ymax   3: (0,-1).x <= -ymin
 * Its id in the `def` output is -1 - s. */
static void box_side(const double box[4], int s, double* gx, double* gy, double* gb) {
    switch (s) {
    case 0: *gx = 1.0;  *gy = 0.0;  *gb = box[1];  break;
    case 1: *gx = -1.0; *gy = 0.0;  *gb = -box[0]; break;
    case 2: *gx = 0.0;  *gy = 1.0;  *gb = box[3];  break;
    default: *gx = 0.0; *gy = -1.0; *gb = -box[2]; break;
    }
}

/* Solve one LP.  box = {xmin, xmax, ymin, ymax}.
 * def[0..2]: the ids that define the result.  OPTIMAL / BOX_BOUNDED: the two
 * constraints through the returned vertex (def[2] = INT32_MIN).  INFEASIBLE: the
 * violated constraint, then the lower and upper endpoint constraints of the empty
 * interval, or the violated constraint and one parallel constraint (def[2] =
 * INT32_MIN).  Ids >= 0 index the LP's own constraints; -1..-4 are the box sides.
 * Returns the status. */
int32_t oracle_solve_lp(const float* ax, const float* ay, const float* b, int64_t m,
                        float cx_f, float cy_f, const double box[4], uint64_t seed,
                        double eps, double* xy, int32_t* def, int64_t* nviol_out) {
    const int32_t NONE = INT32_MIN;
    double cx = (double)cx_f, cy = (double)cy_f;
    int64_t nviol = 0;
    def[0] = def[1] = def[2] = NONE;

    int bad = !isfinite(cx) || !isfinite(cy);
    for (int64_t i = 0; i < m && !bad; i++)
        if (!isfinite(ax[i]) || !isfinite(ay[i]) || !isfinite(b[i])) bad = 1;
    if (bad) {
        xy[0] = xy[1] = NAN;
        if (nviol_out) *nviol_out = 0;
        return ORACLE_BAD_INPUT;
    }

    /* Visit order, materialised once: order[k] = pi(k). */
    int64_t* order = (int64_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    oracle_perm P;
    perm_init(&P, seed, (uint64_t)m);
    visit_order(&P, m, order);

    /* Start at the box corner that maximises c (the optimum of the box alone). */
    double x0 = (cx >= 0.0) ? box[1] : box[0];
    double x1 = (cy >= 0.0) ? box[3] : box[2];
    def[0] = (cx >= 0.0) ? -1 : -2;
    def[1] = (cy >= 0.0) ? -3 : -4;
    int32_t status = -1;

    for (int64_t i = 0; i < m; i++) {
        int64_t h = order[i];
        double hx = (double)ax[h], hy = (double)ay[h], hb = (double)b[h];
        double s = hx * x0 + hy * x1 - hb;
        double tol = eps * (fabs(hx * x0) + fabs(hy * x1) + fabs(hb));
        if (!(s > tol)) continue; /* outcome (1): the optimum satisfies the constraint */

        /* Outcome (2): the new optimum lies on line l: hx*x + hy*y = hb. */
        double nrm2 = hx * hx + hy * hy;
        if (nrm2 == 0.0) { /* 0.x <= hb with hb < 0 */
            def[0] = (int32_t)h; def[1] = NONE; def[2] = NONE;
            status = ORACLE_INFEASIBLE;
            break;
        }
        /* Parameterise l as p0 + t*u, u parallel to l. */
        double p0x = hx * hb / nrm2, p0y = hy * hb / nrm2;
        double ux = -hy, uy = hx;

        double u_left = -INFINITY, u_right = INFINITY;
        int32_t id_left = NONE, id_right = NONE;
        int32_t parallel_bad = NONE;
        /* Earlier constraints in visit-position order: box sides at -4..-1, then
         * positions 0..i-1.  Strict comparisons keep the earliest position on ties. */
        for (int64_t j = -4; j < i; j++) {
            double gx, gy, gb;
            int32_t gid;
            if (j < 0) {
                int side = (int)(j + 4);
                box_side(box, side, &gx, &gy, &gb);
                gid = -1 - side;
            } else {
                int64_t g = order[j];
                gx = (double)ax[g]; gy = (double)ay[g]; gb = (double)b[g];
                gid = (int32_t)g;
            }
            /* g.(p0 + t u) <= gb  <=>  t * (g.u) <= gb - g.p0 */
            double den = gx * ux + gy * uy;
            double num = gb - (gx * p0x + gy * p0y);
            if (den > 0.0) {         /* bounded to the right: Eq. 4 */
                double t = num / den;
                if (t < u_right) { u_right = t; id_right = gid; }
            } else if (den < 0.0) {  /* bounded to the left: Eq. 3 */
                double t = num / den;
                if (t > u_left) { u_left = t; id_left = gid; }
            } else if (num < 0.0) {  /* parallel and excluding the line */
                parallel_bad = gid;
                break;
            }
        }
        nviol++;
        if (parallel_bad != NONE) {
            def[0] = (int32_t)h; def[1] = parallel_bad; def[2] = NONE;
            status = ORACLE_INFEASIBLE;
            break;
        }
        if (u_left > u_right) {
            def[0] = (int32_t)h; def[1] = id_left; def[2] = id_right;
            status = ORACLE_INFEASIBLE;
            break;
        }
        double cu = cx * ux + cy * uy;
        double t;
        int32_t e;
        if (cu > 0.0) { t = u_right; e = id_right; }
        else          { t = u_left;  e = id_left;  }
        x0 = p0x + t * ux;
        x1 = p0y + t * uy;
        def[0] = (int32_t)h; def[1] = e; def[2] = NONE;
    }
    free(order);
    if (nviol_out) *nviol_out = nviol;
    if (status == ORACLE_INFEASIBLE) {
        xy[0] = xy[1] = NAN;
        return status;
    }
    xy[0] = x0;
    xy[1] = x1;
    return (def[0] < 0 || def[1] < 0) ? ORACLE_BOX_BOUNDED : ORACLE_OPTIMAL;
}

/* Solve LPs [lp_begin, lp_end) of a CSR batch.  offsets[l]..offsets[l+1] is LP l's
 * slice of ax/ay/b; obj holds (cx, cy) per LP; seed_l = seed + l.
 * out_xy: 2 doubles per LP (indexed by l), out_status: 1 int per LP, out_def: 3 ints
 * per LP or NULL, out_nviol: 1 int64 per LP or NULL. */
void oracle_solve_batch(const float* ax, const float* ay, const float* b,
                        const int64_t* offsets, int64_t lp_begin, int64_t lp_end,
                        const float* obj, double xmin, double xmax, double ymin,
                        double ymax, uint64_t seed, double eps, double* out_xy,
                        int32_t* out_status, int32_t* out_def, int64_t* out_nviol) {
    double box[4] = {xmin, xmax, ymin, ymax};
    for (int64_t l = lp_begin; l < lp_end; l++) {
        int64_t o = offsets[l];
        int64_t m = offsets[l + 1] - o;
        int32_t def[3];
        int64_t nv = 0;
        int32_t st = oracle_solve_lp(ax + o, ay + o, b + o, m, obj[2 * l], obj[2 * l + 1],
                                     box, seed + (uint64_t)l, eps, out_xy + 2 * l, def, &nv);
        out_status[l] = st;
        if (out_def) {
            out_def[3 * l] = def[0];
            out_def[3 * l + 1] = def[1];
            out_def[3 * l + 2] = def[2];
        }
        if (out_nviol) out_nviol[l] = nv;
    }
}
