// lp2d_persistent.cu -- the persistent, queue-balanced batched Seidel solver.
//
// The paper balances the uneven cost of 1-D LPs by spreading work units over the
// threads of a block (Sec. 3).  Here the balancing happens at the level of whole LPs:
// a grid of (SMs x resident CTAs) persistent CTAs pulls spans of LP indices from three
// device queue heads, one per size class, until all are exhausted.
//   phase 1: LPs with more than kCapMid constraints, one at a time per CTA: the CTA
//            stages the LP in its 24 KB of shared memory, warp 0 runs Seidel's
//            iterations and warps 1..3 join only the long 1-D LPs (LPs above kCapBig
//            are read from global memory in visit order instead);
//   phase 2: LPs with more than kCapSmall and at most kCapMid constraints, one per
//            warp for warps 0 and 1, each with half of the stage (their 1-D LPs are
//            too short for helpers, so two drivers share a CTA's stage);
//   phase 3: LPs with at most kCapSmall constraints, one per warp, each warp with a
//            quarter of the stage;
//   phase 4 (FP32): LPs with at most P.lane_max_m (<= kCapLane) constraints, one per
//            lane, 32 per warp (lp2d_lane.cuh); phase 3 then leaves them out.
// Large LPs therefore start first and small ones fill the tail.  The last CTA to
// finish resets the queue heads, so the workspace is ready for the next launch on
// the same stream without a memset.
#include "lp2d_internal.h"
#include "lp2d_lane.cuh"
#include "lp2d_solve.cuh"
#include "lp2d_warp.cuh"

namespace lp2d {

constexpr int kWarpSlots = kStageSlots / kPersistentWarps;  // stage slots per warp (phase 3)
constexpr int kMidWarps = 2;                                // warps with half a stage each (phase 2)
constexpr int kMidSlots = kStageSlots / kMidWarps;          // their stage slots
static_assert(kWarpSlots - kBoxSlots >= kCapSmall, "quarter-stage capacity");
static_assert(kMidSlots - kBoxSlots >= kCapMid && kCapMid <= 1024, "half-stage capacity (32-word key bitmap)");
static_assert(kStageSlots - kBoxSlots >= kCapBig && kCapBig <= 4096, "stage capacity (128-word key bitmap)");
// Keys a thread keeps in registers between the staging passes (two per register).
constexpr int kKeysSmall = (kCapSmall + 31) / 32;
constexpr int kKeysMid = 0;  // computed again: fewer registers and less code
constexpr int kKeysBig = (kCapBig + 127) / 128;

// Rows of 32 positions the FP32 driver tests per step, per phase: more rows shorten the
// serial chain of an LP, fewer cost fewer instructions.
constexpr int kRowsBig = 2;
constexpr int kRowsMid = 1;
constexpr int kRowsSmall = 1;
static_assert(32 * kLaneCap <= kWarpSlots && kCapLane <= kLaneCap, "32 single-lane LPs fill a warp's stage");

// The FP32 iterations have their own driver (Rows rows of 32 positions per step); the
// other precisions share drive_lp2.
template <typename Real, bool kMixed, bool kTeam, int Rows>
__device__ __forceinline__ void drive(const Params& P, int64_t lp, int m, float cx, float cy, const VisitOrder& vo,
                                      const float2* sA, const float* sB, const unsigned* bm, int lane,
                                      TeamJob2<Real>* job) {
    if constexpr (sizeof(Real) == 4 && !kMixed)
        drive_f32<kTeam, Rows>(P, lp, m, cx, cy, vo, sA, sB, bm, lane, job);
    else
        drive_lp2<Real, kMixed, kTeam>(P, lp, m, cx, cy, vo, sA, sB, bm, lane, job);
}

template <typename Real>
__device__ __forceinline__ void write_bad(const Params& P, int64_t lp) {
    atomicOr(P.ws + kWsError, static_cast<unsigned long long>(kDevErrBadOffsets));
    P.out_status[lp] = kBadInput;
    Real* out = reinterpret_cast<Real*>(P.out_xy);
    out[2 * lp] = out[2 * lp + 1] = real_inf<Real>() - real_inf<Real>();
}

// Span of the next queue grab: a grab that held none of the caller's LPs doubles it
// (up to `cap`), one that held more than `target` of them halves it (down to 1).  A
// class that is rare in the batch thus costs few queue operations, and a dense one
// keeps grabs small enough to balance the load across the grid.
__device__ __forceinline__ int next_span(int span, int found, int target, int cap = 32) {
    if (found == 0) return min(2 * span, cap);
    if (found > target) return max(span >> 1, 1);
    return span;
}

// Largest span of phases 1 and 2, whose classes fill about an eighth of the LP indices
// each: a grab of 32 can hold several of their LPs, which one CTA or warp then solves
// one after another while the others run out of work at the end of the phase.
constexpr int kSpanCapSparse = 16;

// A warp's next grab from the queue at *head: `span` LP indices starting at the
// returned index; lane l < span gets the first offset, the size and the objective of
// LP start + l.  The caller picks its LPs out of the grab by ballot.
__device__ __forceinline__ long long warp_grab(const Params& P, unsigned long long* head, int span, int lane,
                                               long long& off_l, long long& mm_l, float& cx_l, float& cy_l) {
    long long start = 0;
    if (lane == 0) start = static_cast<long long>(atomicAdd(head, static_cast<unsigned long long>(span)));
    start = __shfl_sync(kFull, start, 0);
    off_l = 0;
    mm_l = 0;
    cx_l = cy_l = 0.0f;
    if (start >= 0 && start < P.n_lp && lane < span && start + lane < P.n_lp) {
        off_l = __ldg(P.offsets + start + lane);
        mm_l = __ldg(P.offsets + start + lane + 1) - off_l;
        cx_l = __ldg(P.obj + 2 * (start + lane));
        cy_l = __ldg(P.obj + 2 * (start + lane) + 1);
    }
    return start;
}

// Lanes whose bit is set in `todo` prefetch their LP's constraint segments into L2.
__device__ __forceinline__ void prefetch_grab(const Params& P, unsigned todo, long long off_l, long long mm_l,
                                              int lane) {
    if (P.prefetch && ((todo >> lane) & 1u)) {
        prefetch_l2(P.ax + off_l, mm_l);
        prefetch_l2(P.ay + off_l, mm_l);
        prefetch_l2(P.b + off_l, mm_l);
    }
}

template <typename Real, bool kMixed>
__device__ __forceinline__ void persistent_body(const Params& P) {
    __shared__ float2 sA[kStageSlots];
    __shared__ float sB[kStageSlots];
    __shared__ unsigned s_bm[kPersistentWarps * 32];  // key bitmaps (32 words per warp, 128 per CTA)
    __shared__ int s_pre[kPersistentWarps * 32];      // their prefix counts
    __shared__ int s_wsum[kPersistentWarps];
    __shared__ TeamJob2<Real> job;
    __shared__ TeamScratch<kPersistentWarps> sc;  // the read-from-HBM path
    __shared__ long long s_grab;
    __shared__ long long s_off[kMaxChunk + 1];
    __shared__ float s_obj[2 * kMaxChunk];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    unsigned phase = 0;
    // the largest LP solved by a single lane (FP32 only; 0: none)
    const int tiny = (sizeof(Real) == 4 && !kMixed) ? P.lane_max_m : 0;
    unsigned long long* ws = P.ws;

    // ---- phase 1: large LPs, one CTA each (grab spans adapt as in next_span)
    if (warp == 0) write_box2(P, sA, sB, lane);  // slots 0..3 stay the box for the whole phase
    int big_span = P.chunk_big;
    for (;;) {
        __syncthreads();  // the previous chunk's s_grab / s_off / stage are no longer read
        if (tid == 0) s_grab = static_cast<long long>(atomicAdd(ws + kWsHeadBig, static_cast<unsigned long long>(big_span)));
        __syncthreads();
        const long long start = s_grab;
        if (start < 0 || start >= P.n_lp) break;  // a head past 2^63 is not a valid LP index
        const int cnt = static_cast<int>(min(static_cast<long long>(big_span), P.n_lp - start));
        if (tid <= cnt) s_off[tid] = __ldg(P.offsets + start + tid);
        if (tid < 2 * cnt) s_obj[tid] = __ldg(P.obj + 2 * start + tid);
        __syncthreads();
        if (P.prefetch && tid < cnt) {
            const long long o = s_off[tid], n = s_off[tid + 1] - o;
            if (n > kCapMid && n <= kCapBig) {
                prefetch_l2(P.ax + o, n);
                prefetch_l2(P.ay + o, n);
                prefetch_l2(P.b + o, n);
            }
        }
        int found = 0;
        for (int i = 0; i < cnt; ++i) {
            const int64_t lp = start + i;
            const int64_t base = s_off[i];
            const int64_t mm = s_off[i + 1] - base;
            if (mm <= kCapMid) continue;  // phases 2 and 3 (negative sizes are reported there)
            ++found;
            if (mm > kMaxKeyPathM) {
                if (tid == 0) write_bad<Real>(P, lp);
                continue;
            }
            const int m = static_cast<int>(mm);
            if (m > kCapBig) {
                solve_lp_keys<kPersistentWarps, Real, kMixed>(P, lp, base, m, &sc, phase, tid);
                continue;
            }
            VisitOrder vo;
            warp_visit_order(vo, P.seed + static_cast<uint64_t>(lp), static_cast<uint32_t>(m), lane);
            stage_lp2<128, 128, kKeysBig>(vo, m, P.ax + base, P.ay + base, P.b + base, sA, sB, s_bm, s_pre, s_wsum, tid);
            cp_async_wait_all();
            __syncthreads();
            if (warp == 0)
                drive<Real, kMixed, true, kRowsBig>(P, lp, m, s_obj[2 * i], s_obj[2 * i + 1], vo, sA, sB, s_bm, lane, &job);
            else
                team_helper2<Real, kMixed>(sA, sB, &job, tid);
            __syncthreads();
        }
        big_span = next_span(big_span, found, P.chunk_big, kSpanCapSparse);
    }

    // ---- phase 2: mid-size LPs, one warp each for warps 0 and 1 (half a stage each)
    if (warp < kMidWarps) {
        float2* hA = sA + warp * kMidSlots;
        float* hB = sB + warp * kMidSlots;
        unsigned* hbm = s_bm + warp * 32;
        int* hpre = s_pre + warp * 32;
        write_box2(P, hA, hB, lane);
        int span = P.chunk_small;
        for (;;) {
            long long off_l, mm_l;
            float cx_l, cy_l;
            const long long start = warp_grab(P, ws + kWsHeadMid, span, lane, off_l, mm_l, cx_l, cy_l);
            if (start < 0 || start >= P.n_lp) break;
            unsigned todo = __ballot_sync(kFull, lane < span && mm_l > kCapSmall && mm_l <= kCapMid);
            span = next_span(span, __popc(todo), P.chunk_small, kSpanCapSparse);
            prefetch_grab(P, todo, off_l, mm_l, lane);
            while (todo != 0u) {
                const int i = __ffs(todo) - 1;
                todo &= todo - 1u;
                const int64_t lp = start + i;
                const int64_t base = __shfl_sync(kFull, off_l, i);
                const int m = static_cast<int>(__shfl_sync(kFull, mm_l, i));
                const float cx = __shfl_sync(kFull, cx_l, i), cy = __shfl_sync(kFull, cy_l, i);
                VisitOrder vo;
                warp_visit_order(vo, P.seed + static_cast<uint64_t>(lp), static_cast<uint32_t>(m), lane);
                stage_lp2<32, 32, kKeysMid>(vo, m, P.ax + base, P.ay + base, P.b + base, hA, hB, hbm, hpre, nullptr,
                                            lane);
                cp_async_wait_all();
                __syncwarp();
                drive<Real, kMixed, false, kRowsMid>(P, lp, m, cx, cy, vo, hA, hB, hbm, lane, nullptr);
                __syncwarp();  // all lanes are done with the stage before it is overwritten
            }
        }
    }
    __syncthreads();  // the half stages are free for phase 3

    // ---- phase 3: small LPs, one warp each
    float2* wA = sA + warp * kWarpSlots;
    float* wB = sB + warp * kWarpSlots;
    unsigned* wbm = s_bm + warp * 32;
    int* wpre = s_pre + warp * 32;
    write_box2(P, wA, wB, lane);
    int span = P.chunk_small;
    for (;;) {
        long long off_l, mm_l;
        float cx_l, cy_l;
        const long long start = warp_grab(P, ws + kWsHeadSmall, span, lane, off_l, mm_l, cx_l, cy_l);
        if (start < 0 || start >= P.n_lp) break;
        // negative sizes (bad offsets) are reported here; LPs for single lanes are not
        unsigned todo = __ballot_sync(kFull, lane < span && start + lane < P.n_lp && mm_l <= kCapSmall &&
                                                 !(tiny > 0 && mm_l >= 0 && mm_l <= tiny));
        span = next_span(span, __popc(todo), P.chunk_small);
        prefetch_grab(P, todo, off_l, mm_l, lane);
        while (todo != 0u) {
            const int i = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int64_t lp = start + i;
            const int64_t base = __shfl_sync(kFull, off_l, i);
            const int64_t mm = __shfl_sync(kFull, mm_l, i);
            if (mm < 0) {
                if (lane == 0) write_bad<Real>(P, lp);
                continue;
            }
            const int m = static_cast<int>(mm);
            const float cx = __shfl_sync(kFull, cx_l, i), cy = __shfl_sync(kFull, cy_l, i);
            VisitOrder vo;
            warp_visit_order(vo, P.seed + static_cast<uint64_t>(lp), static_cast<uint32_t>(m), lane);
            stage_lp2<32, 32, kKeysSmall>(vo, m, P.ax + base, P.ay + base, P.b + base, wA, wB, wbm, wpre, nullptr, lane);
            cp_async_wait_all();
            __syncwarp();
            drive<Real, kMixed, false, kRowsSmall>(P, lp, m, cx, cy, vo, wA, wB, wbm, lane, nullptr);
            __syncwarp();  // all lanes are done with the stage before it is overwritten
        }
    }

    // ---- phase 4 (FP32): LPs of at most `tiny` constraints, one lane each, 32 per warp,
    // in the warp's part of the stage (position p of lane l in slot 32 p + l)
    if (tiny > 0) {
        // pending LPs: lane i < np holds the i-th (index, first offset, size, objective);
        // a grab spans only the lanes still free, so the list never overflows
        long long p_lp = 0, p_off = 0;
        int p_m = 0;
        float p_cx = 0.0f, p_cy = 0.0f;
        int np = 0;
        bool more = true;
        for (;;) {
            while (more && np < 32) {
                const int span = 32 - np;
                long long off_l, mm_l;
                float cx_l, cy_l;
                const long long start = warp_grab(P, ws + kWsHeadTiny, span, lane, off_l, mm_l, cx_l, cy_l);
                if (start < 0 || start >= P.n_lp) {
                    more = false;
                    break;
                }
                const unsigned found =
                    __ballot_sync(kFull, lane < span && start + lane < P.n_lp && mm_l >= 0 && mm_l <= tiny);
                const int cnt = __popc(found);
                // lanes np .. np + cnt - 1 take the found LPs in index order
                const int t = lane - np;
                const bool take = t >= 0 && t < cnt;
                const int src = take ? nth_set_bit(found, t) : lane;
                const long long o = __shfl_sync(kFull, off_l, src);
                const long long n = __shfl_sync(kFull, mm_l, src);
                const float ocx = __shfl_sync(kFull, cx_l, src), ocy = __shfl_sync(kFull, cy_l, src);
                if (take) {
                    p_lp = start + src;
                    p_off = o;
                    p_m = static_cast<int>(n);
                    p_cx = ocx;
                    p_cy = ocy;
                }
                np += cnt;
            }
            if (np == 0) break;
            const bool valid = lane < np;
            const int m = valid ? p_m : 0;
            VisitOrder vo;
            vo.init(P.seed + static_cast<uint64_t>(p_lp), static_cast<uint32_t>(m));
            const uint64_t ord = stage_lane(vo, m, P.ax + p_off, P.ay + p_off, P.b + p_off, wA, wB, lane);
            cp_async_wait_all();
            __syncwarp();
            solve_lane_f32(P, p_lp, valid, m, p_cx, p_cy, ord, wA, wB, lane);
            __syncwarp();  // all lanes are done with the stage before it is overwritten
            np = 0;
        }
    }

    // ---- the last CTA out resets the queue heads for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(ws + kWsDone, 1ull);
        if (prev == static_cast<unsigned long long>(gridDim.x) - 1ull) {
            atomicExch(ws + kWsHeadBig, 0ull);
            atomicExch(ws + kWsHeadSmall, 0ull);
            atomicExch(ws + kWsHeadMid, 0ull);
            atomicExch(ws + kWsHeadTiny, 0ull);
            atomicExch(ws + kWsDone, 0ull);
        }
    }
}

// The FP32 kernels are fitted to kPersistentMinCtas resident CTAs per SM (the shared
// memory of a CTA allows that many; registers must not take one away); the FP64 one
// keeps the compiler's register choice.
template <typename Real>
__global__ void __launch_bounds__(kPersistentWarps * 32, sizeof(Real) == 4 ? kPersistentMinCtas : 1)
seidel_persistent_kernel(const Params P) {
    persistent_body<Real, false>(P);
}

__global__ void __launch_bounds__(kPersistentWarps * 32, kPersistentMinCtas)
seidel_persistent_mixed_kernel(const Params P) {
    persistent_body<float, true>(P);
}

cudaError_t launch_persistent_f32(const Params& p, int grid, cudaStream_t s) {
    seidel_persistent_kernel<float><<<grid, kPersistentWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_persistent_mixed(const Params& p, int grid, cudaStream_t s) {
    seidel_persistent_mixed_kernel<<<grid, kPersistentWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_persistent_f64(const Params& p, int grid, cudaStream_t s) {
    seidel_persistent_kernel<double><<<grid, kPersistentWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t persistent_occupancy(int precision, int* ctas_per_sm) {
    const int threads = kPersistentWarps * 32;
    if (precision == 2)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, seidel_persistent_kernel<double>, threads, 0);
    if (precision == 1)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, seidel_persistent_mixed_kernel, threads, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, seidel_persistent_kernel<float>, threads, 0);
}

}  // namespace lp2d
