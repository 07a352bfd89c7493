/*
 * lp3d.h -- C ABI of the batched 3-D linear-program solver.
 *
 * The method of Charlton, Maddock & Richmond (arXiv 1902.04995) one dimension up:
 * the paper gives Seidel's randomized incremental algorithm in two dimensions
 * (Sec. 2.1) and names higher dimensions as the next step (Sec. 6).  Every LP of a
 * batch is
 *
 *     maximise  c^T x   subject to   A x <= b,   x in R^3
 *
 * intersected with a bounding box (six planes).  Constraints are visited in the
 * same seeded random order as the 2-D solver's (see lp2d_visit_order); when the
 * current optimum violates the visited constraint, the new optimum is found on that
 * constraint's plane by a 2-D LP over the box and every earlier constraint, itself
 * solved by Seidel's 2-D method with 1-D LPs on lines (Eqs. 3, 4).
 *
 * Conventions are those of lp2d.h (asynchronous, stream-ordered, caller-owned device
 * memory, lp2d_last_error() for the reason of a non-zero return), with:
 * - constraint i: ax[i]*x + ay[i]*y + az[i]*z <= b[i] (float32, SoA); LP l owns
 *   constraints offsets[l] .. offsets[l+1]-1 (int64 CSR, device);
 * - obj_xyz[3*l .. 3*l+2] = (c_x, c_y, c_z) of LP l (float32, device);
 * - out_xyz[3*l .. 3*l+2]: the optimal vertex (float32; float64 for LP2D_PREC_FP64);
 *   INFEASIBLE and BAD_INPUT LPs get NaN; out_status[l] as in lp2d.h, BOX_BOUNDED when
 *   a box plane is one of the three planes through the vertex;
 * - an LP may have at most LP3D_MAX_CONSTRAINTS constraints: a larger one gets status
 *   LP2D_BAD_INPUT and sets bit LP2D_DEVERR_TOO_LARGE of the workspace error word.
 */
#ifndef LP3D_H
#define LP3D_H

#include "lp2d.h"

#ifdef __cplusplus
extern "C" {
#endif

/** Largest LP the 3-D solver stages: LPs of up to 1018 constraints share a CTA's stage
    (1024 slots less the six box planes per warp); larger ones go to a one-warp kernel
    with a 12288-slot stage in dynamic shared memory (12288 less the six box planes). */
#define LP3D_MAX_CONSTRAINTS 12282

/** The bounding box (finite, min < max on every axis); the box planes have visit
 *  positions -6..-1 in the order x <= xmax, -x <= -xmin, y <= ymax, -y <= -ymin,
 *  z <= zmax, -z <= -zmin, and ids -1..-6 in out_def. */
typedef struct {
    float xmin, xmax, ymin, ymax, zmin, zmax;
} lp3d_box;

/**
 * Solve a batch of 3-D LPs.  Options as for lp2d_solve_batch_ex: precision
 * LP2D_PREC_FP32 or LP2D_PREC_FP64 (LP2D_PREC_FP32_F64ISECT and the uniform schedule
 * give LP2D_ERR_UNSUPPORTED); chunk_small is the target number of LPs per queue grab;
 * out_nviol counts the violations at the top level (each one a 2-D LP); out_def
 * receives three constraint ids per LP.  The workspace is lp2d_workspace_bytes()
 * bytes, zeroed once (lp2d_workspace_init) and reused by later launches on the same
 * stream; it is not capture-safe to share between concurrent launches.
 * Returns an lp2d_err.
 */
int lp3d_solve_batch_ex(const float* ax, const float* ay, const float* az, const float* b,
                        const int64_t* offsets, int64_t n_lp, const float* obj_xyz, lp3d_box box,
                        void* out_xyz, int32_t* out_status, const lp2d_options* opt, void* workspace,
                        size_t workspace_bytes, lp2d_stream_t stream);

/** Bound of the violation variable of lp2d_least_violation: t <= this factor times
 *  the largest |box| coordinate. */
#define LP2D_LEAST_VIOLATION_TMAX_FACTOR 8.0f

/**
 * Least-violation points of the infeasible LPs of a 2-D batch.  The paper's
 * application (Sec. 5, collision avoidance) needs a velocity even when an agent's LP
 * is infeasible, and the paper names, without specifying it, the extra computation
 * this takes.  This entry point uses the usual choice: the point of the box that
 * minimises the largest violation,
 *
 *     minimise t   subject to   ax[i]*x + ay[i]*y - |(ax[i], ay[i])| t <= b[i],
 *                               (x, y) in box,  0 <= t <= tmax,
 *
 * with tmax = LP2D_LEAST_VIOLATION_TMAX_FACTOR * max |box coordinate| -- a 3-D LP in
 * (x, y, t) with objective (0, 0, -1), solved by the 3-D solver (so an LP may have at
 * most LP3D_MAX_CONSTRAINTS constraints).  For a constraint with a unit normal, the
 * violation is the distance of (x, y) outside it.
 *
 * ax, ay, b, offsets, n_lp, box: the 2-D batch as passed to lp2d_solve_batch_ex.
 * status_in: device int32 [n_lp], the statuses of that solve; only LPs with
 * LP2D_INFEASIBLE are solved here, the others' outputs are left untouched.
 * out_xy: device [2*n_lp] (float32; float64 for LP2D_PREC_FP64), the point (x, y) of
 * each solved LP (it may be the 2-D solve's out_xy, to replace the NaNs there).
 * out_t: device float32 [n_lp] or NULL, the least violation t.
 * out_status: device int32 [n_lp], the status of the least-violation LP (OPTIMAL or
 * BOX_BOUNDED: a box plane, which includes t = 0 and t = tmax, defines the point).
 * opt: as for lp3d_solve_batch_ex (seed, precision, out_nviol, out_def refer to
 * the 3-D LP).  Returns an lp2d_err.
 */
int lp2d_least_violation(const float* ax, const float* ay, const float* b, const int64_t* offsets,
                         int64_t n_lp, lp2d_box box, const int32_t* status_in, void* out_xy, float* out_t,
                         int32_t* out_status, const lp2d_options* opt, void* workspace,
                         size_t workspace_bytes, lp2d_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LP3D_H */
