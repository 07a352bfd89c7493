/*
 * lpnd.h -- C ABI of the batched d-dimensional linear-program solver (d = 2..5).
 *
 * The method of Charlton, Maddock & Richmond (arXiv 1902.04995) in up to five
 * dimensions: the paper gives Seidel's randomized incremental algorithm in two
 * dimensions (Sec. 2.1) and names higher dimensions as the next step (Sec. 6).  Every
 * LP of a batch is
 *
 *     maximise  c^T x   subject to   A x <= b,   x in R^d
 *
 * intersected with a bounding box (2d planes).  Constraints are visited in the same
 * seeded random order as the 2-D solver's (see lp2d_visit_order).  When the current
 * optimum violates the visited constraint, the new optimum is found on that
 * constraint's hyperplane by the (d-1)-dimensional LP over the box and every earlier
 * constraint, solved the same way one dimension down, until the 1-D LPs of Eqs. 3
 * and 4; an infeasible lower-dimensional LP makes the LP infeasible.
 *
 * Conventions are those of lp2d.h (asynchronous, stream-ordered, caller-owned device
 * memory, lp2d_last_error() for the reason of a non-zero return), with:
 * - constraint i of the batch: a[0][i]*x_0 + ... + a[d-1][i]*x_{d-1} <= b[i]
 *   (float32, one device array per coefficient); LP l owns constraints offsets[l] ..
 *   offsets[l+1]-1 (int64 CSR, device);
 * - obj[d*l .. d*l+d-1] = c of LP l (float32, device);
 * - out_x[d*l .. d*l+d-1]: the optimal vertex (float32; float64 for LP2D_PREC_FP64);
 *   INFEASIBLE and BAD_INPUT LPs get NaN; out_status[l] as in lp2d.h, BOX_BOUNDED when
 *   a box plane is one of the d planes through the vertex;
 * - an LP may have at most LPND_MAX_CONSTRAINTS(d) constraints: a larger one gets
 *   status LP2D_BAD_INPUT and sets bit LP2D_DEVERR_TOO_LARGE of the workspace error
 *   word.
 */
#ifndef LPND_H
#define LPND_H

#include "lp2d.h"

#ifdef __cplusplus
extern "C" {
#endif

/** Largest dimension the solver is built for. */
#define LPND_MAX_DIM 5

/** Largest LP the d-dimensional solver stages: LPs of up to 1024 - 2d constraints
 *  share a CTA's stage (1024 slots per warp, less the 2d box planes); larger ones go to
 *  a one-warp kernel with an 8192-slot stage in dynamic shared memory. */
#define LPND_MAX_CONSTRAINTS(d) (8192 - 2 * (d))

/**
 * Solve a batch of d-dimensional LPs, 2 <= d <= LPND_MAX_DIM.
 *
 * a:   HOST array of d DEVICE pointers; a[t] is float32 [n_constraints], coefficient
 *      t of every constraint.  The host array is read during the call only.
 * b:   device float32 [n_constraints].
 * box: HOST array of 2d floats {min_0, max_0, min_1, max_1, ...}, finite, min < max on
 *      every axis, read during the call only.  The box planes have visit positions
 *      -2d..-1 in the order x_0 <= max_0, -x_0 <= -min_0, x_1 <= max_1, ... and ids
 *      -1..-2d in out_def.
 * Options as for lp2d_solve_batch_ex: precision LP2D_PREC_FP32 or LP2D_PREC_FP64
 * (LP2D_PREC_FP32_F64ISECT and the uniform schedule give LP2D_ERR_UNSUPPORTED);
 * chunk_small is the target number of LPs per queue grab (0: 2); out_nviol counts
 * the violations in the whole space (each one a (d-1)-dimensional LP); out_def
 * receives d constraint ids per LP (INT32_MIN for INFEASIBLE and BAD_INPUT LPs).  The
 * workspace is lp2d_workspace_bytes() bytes, zeroed once (lp2d_workspace_init) and
 * reused by later launches on the same stream; it is not safe to share between
 * concurrent launches.
 * Returns an lp2d_err: LP2D_ERR_INVALID_ARGUMENT for d outside 2..LPND_MAX_DIM, a
 * NULL or misaligned pointer, a bad box or n_lp < 0; nothing is launched then.
 */
int lpnd_solve_batch(int d, const float* const* a, const float* b, const int64_t* offsets, int64_t n_lp,
                     const float* obj, const float* box, void* out_x, int32_t* out_status,
                     const lp2d_options* opt, void* workspace, size_t workspace_bytes, lp2d_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LPND_H */
