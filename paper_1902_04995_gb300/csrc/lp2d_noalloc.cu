// lp2d_noalloc.cu -- lp2d_solve_batch_noalloc: the persistent solve without any
// device allocation.
//
// Some callers cannot allocate device memory at all.  Examples: a plugin inside a host
// framework that owns every device byte through its own pool and forbids direct
// cudaMalloc; a real-time loop that must not allocate once running, because cudaMalloc
// can synchronise the device and stall it; a caller in another language that has no
// device allocator at hand.
//
// This entry point needs nothing from them beyond the inputs and outputs.  The queue
// scratch that the persistent kernel uses -- normally the caller's workspace, or a pool
// the library allocates for lp2d_solve_batch -- lives in a fixed device array in this
// file instead.  The loaded library keeps that array on every GPU that loads it until
// the process exits.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "lp2d.h"
#include "lp2d_internal.h"

namespace {

// Largest workspace the array can stand in for (every option set of this library
// needs lp2d_workspace_bytes() == 256 bytes).
constexpr size_t kNoallocScratchBytes = 256;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocScratchBytes / 8];

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int lp2d_solve_batch_noalloc(const float* ax, const float* ay, const float* b, const int64_t* offsets,
                                        int64_t n_lp, const float* obj_xy, lp2d_box box, void* out_xy,
                                        int32_t* out_status, const lp2d_options* opt, lp2d_stream_t stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lp2d::report_error(LP2D_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return lp2d::report_error(LP2D_ERR_UNSUPPORTED, "device %d is beyond the %d devices supported", dev, kMaxDevices);

    const size_t need = lp2d_workspace_bytes(n_lp, opt);
    if (need > kNoallocScratchBytes)
        return lp2d::report_error(LP2D_ERR_UNSUPPORTED,
                                  "lp2d_solve_batch_noalloc: these options need %zu bytes of scratch, more than its "
                                  "fixed %zu-byte device array", need, kNoallocScratchBytes);

    // Set-up, once per device with that device current: the array's name is a host-side
    // stand-in in host code, so the kernel gets the device address from the runtime.
    // The cached address belongs to the device's current context: after a
    // cudaDeviceReset it is stale, and the process must not call this entry point on
    // that device again.
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return lp2d::report_error(LP2D_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s",
                                          cudaGetErrorString(e));
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }

    if (n_lp > 0) {
        // Every call shares the array and finds the last call's contents there: the
        // queue heads, the done counter and the error word must start at zero.
        e = cudaMemsetAsync(scratch, 0, kNoallocScratchBytes, reinterpret_cast<cudaStream_t>(stream));
        if (e != cudaSuccess)
            return lp2d::report_error(LP2D_ERR_CUDA, "clearing the scratch array: %s", cudaGetErrorString(e));
    }
    return lp2d_solve_batch_ex(ax, ay, b, offsets, n_lp, obj_xy, box, out_xy, out_status, opt, scratch,
                               kNoallocScratchBytes, stream);
}
