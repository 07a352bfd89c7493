/*
 * lp2d.h -- C ABI of the GB300 batched 2-D linear-program solver.
 *
 * Method: Charlton, Maddock & Richmond, "Two-Dimensional Batch Linear Programming
 * on the GPU" (arXiv 1902.04995).  Every LP of a batch is
 *
 *     maximise  c^T x   subject to   A x <= b,   x in R^2          (Sec. 2.1, Eq. 1, Eq. 2)
 *
 * intersected with a bounding box (the +-M constraints of Sec. 2.1), and is solved by
 * Seidel's randomized incremental algorithm (Sec. 2.1): constraints are visited in a
 * seeded random order; when the current optimum violates the visited constraint,
 * the new optimum is found on that constraint's line by a 1-D LP over every earlier
 * constraint (Eq. 3 and Eq. 4: a max over left bounds and a min over right bounds).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named "device" are CUDA device (or managed) memory owned by the caller.
 *   The library never frees or retains them beyond the call's stream work.
 * - Calls are asynchronous and ordered on `stream` (a cudaStream_t; NULL is the
 *   legacy default stream).  A non-zero return means nothing was enqueued, and
 *   lp2d_last_error() describes why (thread-local).
 * - Constraint layout (SoA, float32): constraint i is ax[i]*x + ay[i]*y <= b[i].
 *   LP l owns constraints offsets[l] .. offsets[l+1]-1 (CSR, int64, non-decreasing;
 *   offsets[0] need not be 0).  The caller guarantees offsets[n_lp] does not run past
 *   the ends of ax/ay/b.  An LP with negative size gets status LP2D_BAD_INPUT and
 *   sets bit LP2D_DEVERR_BAD_OFFSETS of the workspace error word.
 * - Objectives: obj_xy[2*l], obj_xy[2*l+1] = (c_x, c_y) of LP l, float32.
 * - Visit order of LP l: a permutation pi_l of 0..m_l-1 seeded with seed + l
 *   (uint64 wrap-around); see lp2d_visit_order().  Results of generic LPs do not
 *   depend on the order; the number of 1-D LPs does.
 * - Per-LP results: out_status[l] (int32) and out_xy[2*l..2*l+1], the optimal
 *   vertex (float32 for the FP32 precisions, float64 for LP2D_PREC_FP64).
 *   INFEASIBLE and BAD_INPUT LPs get xy = (NaN, NaN).  An LP with no constraints
 *   returns the box corner that maximises c, with status BOX_BOUNDED.
 */
#ifndef LP2D_H
#define LP2D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/** CUDA stream handle; identical to cudaStream_t. */
typedef struct CUstream_st* lp2d_stream_t;

/** Per-LP outcome written to out_status. */
typedef enum {
    LP2D_OPTIMAL = 0,     /**< vertex defined by two of the LP's own constraints */
    LP2D_INFEASIBLE = 1,  /**< the 1-D LP interval became empty (Eq. 3 > Eq. 4), or a
                               parallel constraint excluded the line (Sec. 2.1) */
    LP2D_BOX_BOUNDED = 2, /**< a side of the bounding box passes through the vertex */
    LP2D_BAD_INPUT = 3    /**< NaN/Inf in the LP's data, or a negative size */
} lp2d_lp_status;

/** Return codes of the entry points. */
typedef enum {
    LP2D_OK = 0,
    LP2D_ERR_INVALID_ARGUMENT = -1,
    LP2D_ERR_CUDA = -2,
    LP2D_ERR_TIMEOUT = -3,       /* reserved: no kernel of this version waits on a flag or a
                                    peer, so no path returns it */
    LP2D_ERR_WORKSPACE = -4,
    LP2D_ERR_UNSUPPORTED = -5
} lp2d_err;

/** Bits of the device error word kept in the workspace. */
enum {
    LP2D_DEVERR_BAD_OFFSETS = 1, /**< an LP had a negative size (status BAD_INPUT) */
    LP2D_DEVERR_TOO_LARGE = 4    /**< a 3-D LP had more than LP3D_MAX_CONSTRAINTS constraints, or a
                                      d-dimensional one more than LPND_MAX_CONSTRAINTS(d) (BAD_INPUT) */
};

/** The bounding box: the +-M constraints of Sec. 2.1 (xmin < xmax, ymin < ymax, finite). */
typedef struct {
    float xmin, xmax, ymin, ymax;
} lp2d_box;

/** Arithmetic of the solve. */
typedef enum {
    LP2D_PREC_FP32 = 0,          /**< FP32 throughout; out_xy is float[2*n_lp] */
    LP2D_PREC_FP32_F64ISECT = 1, /**< FP32, but a 1-D LP work unit whose two normals are
                                      near-parallel (|det| < tau*|a||a_h|) is computed in
                                      FP64; out_xy is float[2*n_lp] */
    LP2D_PREC_FP64 = 2           /**< FP64 arithmetic on the FP32 inputs; out_xy is double[2*n_lp] */
} lp2d_precision;

/** How LPs are mapped to the GPU. */
typedef enum {
    LP2D_SCHED_PERSISTENT = 0, /**< persistent CTAs pull LPs from a device queue; each LP is
                                    staged in shared memory in visit order and solved by a
                                    warp (or a 4-warp team for large LPs) */
    LP2D_SCHED_UNIFORM = 1     /**< one thread per LP, constraints read from global memory
                                    in visit order (the paper's naive mapping, Sec. 3) */
} lp2d_schedule;

/** Options for lp2d_solve_batch_ex.  Fill with lp2d_default_options() first. */
typedef struct {
    uint64_t seed;          /**< seed_l = seed + l; default 0 */
    int32_t precision;      /**< lp2d_precision; default LP2D_PREC_FP32 */
    int32_t schedule;       /**< lp2d_schedule; default LP2D_SCHED_PERSISTENT */
    int32_t ctas_per_sm;    /**< persistent grid = SMs x this; 0 = occupancy maximum */
    int32_t chunk_big;      /**< target large LPs per queue grab by a CTA (1..32); 0 = default 1 */
    int32_t chunk_small;    /**< target LPs per queue grab by a warp (1..16); 0 = default 2 */
    int32_t check_finite;   /**< non-zero: NaN/Inf data gives LP2D_BAD_INPUT; default 1 */
    float eps;              /**< relative violation tolerance; 0 = 1e-6 (FP32) / 1e-12 (FP64) */
    float near_parallel_tau;/**< threshold of LP2D_PREC_FP32_F64ISECT; 0 = 1e-3 */
    int32_t* out_nviol;     /**< optional device int32[n_lp]: number of 1-D LPs solved */
    int32_t* out_def;       /**< optional device int32[2*n_lp]: ids of the two constraints
                                 through the returned vertex (>= 0: the LP's own constraint
                                 index; -1..-4: box side x<=xmax, x>=xmin, y<=ymax, y>=ymin).
                                 Undefined for INFEASIBLE / BAD_INPUT LPs. */
    int32_t team_min_slots; /**< persistent schedule: a 1-D LP of a large LP (more than 1024
                                 constraints) over at least this many earlier constraints (box
                                 included) is shared by the CTA's 128 threads, a shorter one runs
                                 on the driving warp's 32 (64..4096; 0 = default 1024) */
    int32_t l2_prefetch;    /**< persistent schedule: 1 = bulk-prefetch the constraints of every
                                 LP a CTA or warp takes from the queue into L2; 0 (default) or
                                 -1 = no prefetch */
    int32_t lane_max_m;     /**< persistent schedule, LP2D_PREC_FP32: an LP of at most this many
                                 constraints is solved by a single thread, 32 LPs per warp, from
                                 shared memory (threads per LP 1 instead of 32; the results are
                                 bit-identical); 1..16; 0 = default 16; -1 = every LP gets a
                                 whole warp.  Ignored by the other precisions and schedules. */
} lp2d_options;

/** Fill *opt with the defaults listed above. */
void lp2d_default_options(lp2d_options* opt);

/**
 * Bytes of device workspace lp2d_solve_batch_ex takes for this batch size and these
 * options.  The workspace holds the persistent queue heads and the device error
 * word; LP2D_SCHED_UNIFORM runs without one (workspace may be NULL) and then reports
 * bad offsets only through the per-LP status.  It must be zeroed once before its first use
 * (lp2d_workspace_init); every solve leaves it zeroed again, except the error word,
 * which accumulates until read by lp2d_read_device_error.  Two solves that run at
 * the same time must not share a workspace.
 */
size_t lp2d_workspace_bytes(int64_t n_lp, const lp2d_options* opt);
/* (The size depends on neither the batch nor the constraint count -- the workspace is
 * the queue heads and the error word -- so, unlike a size query that also takes the
 * number of constraints, this one takes the LP count only.) */

/** Zero `bytes` of workspace on `stream` (cudaMemsetAsync).  Returns an lp2d_err. */
int lp2d_workspace_init(void* workspace, size_t bytes, lp2d_stream_t stream);

/**
 * Solve a batch with default options (seed 0, FP32, persistent schedule).
 *
 * ax, ay, b:   device float32[offsets[n_lp]]   constraints, SoA
 * offsets:     device int64[n_lp + 1]          CSR row pointers
 * n_lp:        number of LPs (0: nothing is enqueued, returns LP2D_OK)
 * obj_xy:      device float32[2*n_lp]          objective per LP
 * box:         bounding box (by value)
 * out_xy:      device float32[2*n_lp]          optimal vertex per LP
 * out_status:  device int32[n_lp]              lp2d_lp_status per LP
 *
 * The queue workspace comes from a small per-(device, stream) pool that the library
 * allocates on the first call for that stream, so the first call on a stream must
 * not be inside CUDA-graph capture; lp2d_solve_batch_ex with a caller workspace has
 * no such restriction.  Returns an lp2d_err.
 */
int lp2d_solve_batch(const float* ax, const float* ay, const float* b, const int64_t* offsets,
                     int64_t n_lp, const float* obj_xy, lp2d_box box, float* out_xy,
                     int32_t* out_status, lp2d_stream_t stream);

/**
 * Solve a batch with explicit options and a caller-owned workspace (device memory of
 * at least lp2d_workspace_bytes(n_lp, opt) bytes, 8-byte aligned, zeroed once by
 * lp2d_workspace_init; optional for LP2D_SCHED_UNIFORM).  Allocates nothing.
 * out_xy is float32[2*n_lp] for the FP32 precisions and float64[2*n_lp] for
 * LP2D_PREC_FP64.  opt == NULL means the defaults.  Returns an lp2d_err.
 */
int lp2d_solve_batch_ex(const float* ax, const float* ay, const float* b, const int64_t* offsets,
                        int64_t n_lp, const float* obj_xy, lp2d_box box, void* out_xy,
                        int32_t* out_status, const lp2d_options* opt, void* workspace,
                        size_t workspace_bytes, lp2d_stream_t stream);

/**
 * Solve a batch like lp2d_solve_batch_ex, for callers that cannot allocate device
 * memory (a plugin whose host framework owns every device byte, a real-time loop
 * that must not allocate once running, a caller with no device allocator at hand).
 * The paper has no counterpart: this entry point is an interface convenience.
 *
 * The caller passes only inputs and outputs, as in lp2d_solve_batch_ex.  The queue
 * scratch is a fixed 256-byte array in the library's device memory, which every GPU
 * that loads the library keeps until the process exits.  No call of this entry point
 * calls cudaMalloc, cudaFree or any allocating routine.
 * - The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current and keeps it.  Make that first
 *   call before any stream capture.  The kept address dies with the device's
 *   context: after cudaDeviceReset, do not call this entry point on that device
 *   again in the same process.
 * - Every call clears the array on `stream` before its solve.  All calls share the
 *   one array, so calls whose work overlaps on the GPU (other streams, other host
 *   threads) race: order them on one stream, or use lp2d_solve_batch_ex with separate
 *   workspaces.
 * - Options whose workspace exceeds the 256-byte array are rejected with
 *   LP2D_ERR_UNSUPPORTED (none of this version's options do).
 * - Device errors show only in the per-LP status (the error word is not readable).
 *   A non-OK return may still have enqueued the clearing of the library's own array;
 *   no caller memory is touched.
 * Returns an lp2d_err.
 */
int lp2d_solve_batch_noalloc(const float* ax, const float* ay, const float* b, const int64_t* offsets,
                             int64_t n_lp, const float* obj_xy, lp2d_box box, void* out_xy,
                             int32_t* out_status, const lp2d_options* opt, lp2d_stream_t stream);

/**
 * Solve a batch whose inputs and outputs live in host memory (pinned memory gives
 * full copy bandwidth; pageable memory works through staging copies).  The batch
 * is cut at LP boundaries into chunks that shrink towards the end of the batch
 * (40, 30, 17, 9 and 4 % of the last 160M constraints, equal chunks of at most 64M
 * constraints before that; a batch below 2M constraints stays whole).  The chunks
 * are copied to two library-owned device slots on a library copy stream, so that
 * copying chunk i+1 overlaps the solve of chunk i on `stream`; the call then costs
 * about the copy of the whole batch plus the solve of the last, small chunk.  Each
 * chunk's results are copied back on `stream` right after its solve.
 *
 * Arguments are as for lp2d_solve_batch_ex, in host memory: offsets must be host
 * readable, non-decreasing and >= 0 (checked on the host: LP2D_ERR_INVALID_ARGUMENT
 * before anything is enqueued).  out_xy is float32[2*n_lp] (float64 for
 * LP2D_PREC_FP64).  opt->out_nviol / out_def are not supported
 * (LP2D_ERR_UNSUPPORTED).  Each chunk is solved with seed + (index of its first LP),
 * so results equal those of one lp2d_solve_batch_ex call over the whole batch.
 *
 * On return the work is enqueued.  `stream` is ordered after the last copy-out, so
 * synchronising `stream` makes the results readable.  The device slots are
 * allocated on the first call for a (device, stream) pair and grown when a larger
 * chunk needs them, so such a call must not be inside CUDA-graph capture.  Calls on
 * one (device, stream) pair share the slots; the library serialises them with a
 * lock, so a second host thread waits until the first call has enqueued its work.
 * Returns an lp2d_err.
 */
int lp2d_solve_batch_host(const float* ax, const float* ay, const float* b, const int64_t* offsets,
                          int64_t n_lp, const float* obj_xy, lp2d_box box, void* out_xy,
                          int32_t* out_status, const lp2d_options* opt, lp2d_stream_t stream);

/**
 * Write the visit order pi of one LP with m constraints and seed seed_l (the seed of
 * LP l is seed + l) into device int64 out[m]: out[k] is the index of the constraint
 * visited at step k.  Runs the same device code the solver uses (Sec. 2.1 asks for a
 * random visit order; the constraints are visited in increasing order of their keys
 * under a 4-round balanced Feistel network on 2*ceil(ceil(log2 m)/2) bits, at least 2,
 * with SplitMix64 round keys).  m <= 2^26; one CTA.  Returns an lp2d_err.
 */
int lp2d_visit_order(uint64_t seed_l, int64_t m, int64_t* out, lp2d_stream_t stream);

/**
 * Autotune the persistent schedule for a batch: solve it with each candidate of a
 * small grid -- ctas_per_sm in {the occupancy limit, one less}, chunk_big in
 * {1, 2, 4}, chunk_small in {1, 2, 4, 8}, team_min_slots (threads per 1-D LP of a
 * CTA-staged LP: 128 from 512 or 1024 slots on, or always 32) in {512, 1024, 4096},
 * lane_max_m (threads per LP: 1 up to this size, 32 above) in {-1, 8, 16} --
 * timing `reps` solves per candidate with CUDA events on `stream` after one warm-up
 * solve, and write the fastest into opt->ctas_per_sm / chunk_big / chunk_small /
 * team_min_slots / lane_max_m (the other fields of *opt are the base
 * options of every trial; out_nviol / out_def are not written).  The tuned fields
 * change only the speed: results are the same for every setting.  The arguments
 * are those of lp2d_solve_batch_ex; out_xy / out_status hold the last trial's
 * results.  Synchronises `stream`; not for use inside CUDA-graph capture.
 * out_best_ms (host, may be NULL) receives the winner's time per solve.
 * Returns an lp2d_err (LP2D_ERR_UNSUPPORTED for the uniform schedule).
 */
int lp2d_autotune(const float* ax, const float* ay, const float* b, const int64_t* offsets,
                  int64_t n_lp, const float* obj_xy, lp2d_box box, void* out_xy, int32_t* out_status,
                  lp2d_options* opt, void* workspace, size_t workspace_bytes, int reps,
                  float* out_best_ms, lp2d_stream_t stream);

/**
 * Synchronise `stream`, return the device error word accumulated in `workspace`
 * (LP2D_DEVERR_* bits) through *out_bits, and clear it.  Returns an lp2d_err.
 * (The error word lives in the caller's workspace, not in per-stream library state,
 * so the call names the workspace as well as the stream.)
 */
int lp2d_read_device_error(void* workspace, lp2d_stream_t stream, uint32_t* out_bits);

/** Message for the last non-OK return on this thread ("" if none). */
const char* lp2d_last_error(void);

/** Library version string. */
const char* lp2d_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LP2D_H */
