// lp2d_persistent.cu -- the persistent, queue-balanced batched Seidel solver.
//
// The paper balances the uneven cost of 1-D LPs by spreading work units over the
// threads of a block (Sec. 3).  Here the balancing happens at the level of whole LPs:
// a grid of (SMs x resident CTAs) persistent CTAs pulls LP indices from two device
// queue heads until both are exhausted.
//   phase 1: LPs with more than kCapSmall constraints, one at a time per CTA, solved
//            by all 4 warps as a team (staged in the CTA's 24 KB of shared memory;
//            LPs above kCapBig read through the visit order from global memory);
//   phase 2: LPs with at most kCapSmall constraints, one per warp, each warp with
//            its own quarter of the stage.
// Big LPs therefore start first and small ones fill the tail.  The last CTA to
// finish resets the queue heads, so the workspace is ready for the next launch
// on the same stream without a memset.
#include "lp2d_internal.h"
#include "lp2d_solve.cuh"

namespace lp2d {

template <typename Real>
__global__ void __launch_bounds__(kPersistentWarps * 32)
seidel_persistent_kernel(const Params P) {
    __shared__ float sX[kCapBig];
    __shared__ float sY[kCapBig];
    __shared__ float sB[kCapBig];
    __shared__ TeamScratch<kPersistentWarps> sc;
    __shared__ long long s_grab;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    unsigned phase = 0;
    unsigned long long* ws = P.ws;

    // ---- phase 1: large LPs, one CTA team each
    for (;;) {
        __syncthreads();  // everyone has read the previous s_grab
        if (tid == 0) s_grab = static_cast<long long>(atomicAdd(ws + kWsHeadBig, static_cast<unsigned long long>(P.chunk_big)));
        __syncthreads();
        const long long start = s_grab;
        if (start >= P.n_lp) break;
        const long long end = min(start + static_cast<long long>(P.chunk_big), static_cast<long long>(P.n_lp));
        for (long long lp = start; lp < end; ++lp) {
            const int64_t base = __ldg(P.offsets + lp);
            const int64_t m = __ldg(P.offsets + lp + 1) - base;
            if (m <= kCapSmall) continue;  // phase 2 (negative sizes are reported there)
            if (m > 0x7fffffffll) {
                if (tid == 0) {
                    atomicOr(ws + kWsError, static_cast<unsigned long long>(kDevErrBadOffsets));
                    P.out_status[lp] = kBadInput;
                    Real* out = reinterpret_cast<Real*>(P.out_xy);
                    out[2 * lp] = out[2 * lp + 1] = real_inf<Real>() - real_inf<Real>();
                }
                continue;
            }
            if (m <= kCapBig)
                solve_lp<kPersistentWarps, Real, true>(P, lp, base, static_cast<int>(m), sX, sY, sB, &sc, phase, tid);
            else
                solve_lp<kPersistentWarps, Real, false>(P, lp, base, static_cast<int>(m), nullptr, nullptr, nullptr, &sc, phase, tid);
        }
    }

    // ---- phase 2: small LPs, one warp each
    float* wX = sX + warp * kCapSmall;
    float* wY = sY + warp * kCapSmall;
    float* wB = sB + warp * kCapSmall;
    unsigned wphase = 0;
    for (;;) {
        long long start = 0;
        if (lane == 0) start = static_cast<long long>(atomicAdd(ws + kWsHeadSmall, static_cast<unsigned long long>(P.chunk_small)));
        start = __shfl_sync(kFull, start, 0);
        if (start >= P.n_lp) break;
        const long long end = min(start + static_cast<long long>(P.chunk_small), static_cast<long long>(P.n_lp));
        for (long long lp = start; lp < end; ++lp) {
            const int64_t base = __ldg(P.offsets + lp);
            const int64_t m = __ldg(P.offsets + lp + 1) - base;
            if (m > kCapSmall) continue;
            if (m < 0) {
                if (lane == 0) {
                    atomicOr(ws + kWsError, static_cast<unsigned long long>(kDevErrBadOffsets));
                    P.out_status[lp] = kBadInput;
                    Real* out = reinterpret_cast<Real*>(P.out_xy);
                    out[2 * lp] = out[2 * lp + 1] = real_inf<Real>() - real_inf<Real>();
                }
                continue;
            }
            solve_lp<1, Real, true>(P, lp, base, static_cast<int>(m), wX, wY, wB, nullptr, wphase, lane);
            __syncwarp();  // all lanes are done with the stage before it is overwritten
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
            atomicExch(ws + kWsDone, 0ull);
        }
    }
}

cudaError_t launch_persistent_f32(const Params& p, int grid, cudaStream_t s) {
    seidel_persistent_kernel<float><<<grid, kPersistentWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_persistent_f64(const Params& p, int grid, cudaStream_t s) {
    seidel_persistent_kernel<double><<<grid, kPersistentWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t persistent_occupancy(bool fp64, int* ctas_per_sm) {
    if (fp64)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, seidel_persistent_kernel<double>,
                                                             kPersistentWarps * 32, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, seidel_persistent_kernel<float>,
                                                         kPersistentWarps * 32, 0);
}

}  // namespace lp2d
