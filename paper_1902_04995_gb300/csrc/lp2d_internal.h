// lp2d_internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "lp2d_device.cuh"

namespace lp2d {

// Shapes of the persistent schedule (see lp2d_persistent.cu).
constexpr int kPersistentWarps = 4;   // warps per CTA
constexpr int kPersistentMinCtas = 8; // resident CTAs per SM the FP32 register budget is fitted to
constexpr int kStageSlots = 2064;     // stage slots per CTA (8 B + 4 B each)
constexpr int kCapSmall = 512;        // largest LP one warp stages in a quarter of the stage (516 slots)
constexpr int kCapMid = 1024;         // largest LP one warp stages in half of the stage (its keys fit 32 words)
constexpr int kCapBig = 2060;         // largest LP the CTA stages (the box and 2060 constraints)
constexpr int kDefaultTeamMin = 1024; // 1-D LPs over at least this many slots get the helper warps
constexpr int kCapLane = 16;          // largest LP one lane solves alone (32 per warp stage)
constexpr int kDefaultLaneMax = 16;   // default largest LP solved by one lane (FP32)
constexpr int kMaxChunk = 32;         // LP indices per queue grab, at most
constexpr int kMaxChunkSmall = 16;    // largest target of LPs per warp grab
constexpr int kDefaultChunkBig = 1;   // target large LPs per CTA grab
constexpr int kDefaultChunkSmall = 2; // target LPs per warp grab

// Launchers.  Each returns the cudaError_t of the launch.
cudaError_t launch_persistent_f32(const Params& p, int grid, cudaStream_t s);
cudaError_t launch_persistent_f64(const Params& p, int grid, cudaStream_t s);
cudaError_t launch_persistent_mixed(const Params& p, int grid, cudaStream_t s);
cudaError_t launch_uniform_f32(const Params& p, cudaStream_t s);
cudaError_t launch_uniform_f64(const Params& p, cudaStream_t s);
cudaError_t launch_visit_order(uint64_t seed, int64_t m, int64_t* out, cudaStream_t s);

// Resident CTAs per SM of the persistent kernels (occupancy calculator).
cudaError_t persistent_occupancy(int precision, int* ctas_per_sm);

// Record a message for lp2d_last_error() on this thread and return `code`.
int report_error(int code, const char* fmt, ...);

}  // namespace lp2d
