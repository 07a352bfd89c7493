// lp2d_api.cu -- the extern "C" entry points declared in include/lp2d.h: argument
// validation, option defaults, workspace handling and kernel dispatch.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "lp2d.h"
#include "lp2d_internal.h"

namespace {

thread_local char g_last_error[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int ok() {
    g_last_error[0] = '\0';
    return LP2D_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

struct DeviceInfo {
    int sms = 0;
    int occ[3] = {0, 0, 0};  // resident persistent CTAs per SM, per lp2d_precision
};

std::mutex g_mu;
std::map<int, DeviceInfo> g_devices;
std::map<std::pair<int, cudaStream_t>, void*> g_stream_ws;

int device_info(DeviceInfo* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_devices.find(dev);
    if (it != g_devices.end()) {
        *out = it->second;
        return LP2D_OK;
    }
    DeviceInfo info;
    e = cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "SM count: %s", cudaGetErrorString(e));
    for (int prec = 0; prec < 3; ++prec) {
        e = lp2d::persistent_occupancy(prec, &info.occ[prec]);
        if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "occupancy (precision %d): %s", prec, cudaGetErrorString(e));
        if (info.occ[prec] < 1) return fail(LP2D_ERR_CUDA, "persistent kernel cannot be resident");
    }
    g_devices[dev] = info;
    *out = info;
    return LP2D_OK;
}

bool finite(float v) { return std::isfinite(v); }

}  // namespace

namespace lp2d {

int report_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

}  // namespace lp2d

extern "C" {

void lp2d_default_options(lp2d_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->seed = 0;
    opt->precision = LP2D_PREC_FP32;
    opt->schedule = LP2D_SCHED_PERSISTENT;
    opt->ctas_per_sm = 0;
    opt->chunk_big = 0;
    opt->chunk_small = 0;
    opt->check_finite = 1;
    opt->eps = 0.0f;
    opt->near_parallel_tau = 0.0f;
    opt->out_nviol = nullptr;
    opt->out_def = nullptr;
    opt->team_min_slots = 0;
    opt->l2_prefetch = 0;
    opt->lane_max_m = 0;
}

size_t lp2d_workspace_bytes(int64_t n_lp, const lp2d_options* opt) {
    (void)n_lp;
    (void)opt;
    return sizeof(unsigned long long) * lp2d::kWsWords;
}

int lp2d_workspace_init(void* workspace, size_t bytes, lp2d_stream_t stream) {
    if (bytes == 0) return ok();
    if (!workspace) return fail(LP2D_ERR_INVALID_ARGUMENT, "workspace is NULL");
    cudaError_t e = cudaMemsetAsync(workspace, 0, bytes, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    return ok();
}

int lp2d_solve_batch_ex(const float* ax, const float* ay, const float* b, const int64_t* offsets,
                        int64_t n_lp, const float* obj_xy, lp2d_box box, void* out_xy,
                        int32_t* out_status, const lp2d_options* opt_in, void* workspace,
                        size_t workspace_bytes, lp2d_stream_t stream) {
    lp2d_options opt;
    if (opt_in) opt = *opt_in;
    else lp2d_default_options(&opt);

    if (n_lp < 0) return fail(LP2D_ERR_INVALID_ARGUMENT, "n_lp = %lld < 0", (long long)n_lp);
    if (opt.precision < LP2D_PREC_FP32 || opt.precision > LP2D_PREC_FP64)
        return fail(LP2D_ERR_INVALID_ARGUMENT, "unknown precision %d", opt.precision);
    if (opt.schedule != LP2D_SCHED_PERSISTENT && opt.schedule != LP2D_SCHED_UNIFORM)
        return fail(LP2D_ERR_INVALID_ARGUMENT, "unknown schedule %d", opt.schedule);
    if (opt.ctas_per_sm < 0 || opt.chunk_big < 0 || opt.chunk_small < 0)
        return fail(LP2D_ERR_INVALID_ARGUMENT, "negative tuning parameter");
    if (opt.team_min_slots != 0 && (opt.team_min_slots < 64 || opt.team_min_slots > 4096))
        return fail(LP2D_ERR_INVALID_ARGUMENT, "team_min_slots = %d outside 64..4096 (0 = default)",
                    opt.team_min_slots);
    if (opt.l2_prefetch < -1 || opt.l2_prefetch > 1)
        return fail(LP2D_ERR_INVALID_ARGUMENT, "l2_prefetch = %d is not -1, 0 or 1", opt.l2_prefetch);
    if (opt.lane_max_m < -1 || opt.lane_max_m > lp2d::kCapLane)
        return fail(LP2D_ERR_INVALID_ARGUMENT, "lane_max_m = %d outside -1..%d (0 = default, -1 = none)",
                    opt.lane_max_m, lp2d::kCapLane);
    if (!(opt.eps >= 0.0f) || !finite(opt.eps) || !(opt.near_parallel_tau >= 0.0f) || !finite(opt.near_parallel_tau))
        return fail(LP2D_ERR_INVALID_ARGUMENT, "eps / near_parallel_tau must be finite and >= 0");
    if (!finite(box.xmin) || !finite(box.xmax) || !finite(box.ymin) || !finite(box.ymax) ||
        !(box.xmin < box.xmax) || !(box.ymin < box.ymax))
        return fail(LP2D_ERR_INVALID_ARGUMENT, "box must be finite with xmin < xmax and ymin < ymax");
    if (opt.precision == LP2D_PREC_FP32_F64ISECT && opt.schedule == LP2D_SCHED_UNIFORM)
        return fail(LP2D_ERR_UNSUPPORTED, "LP2D_PREC_FP32_F64ISECT needs LP2D_SCHED_PERSISTENT");
    if (n_lp == 0) return ok();
    if (!ax || !ay || !b || !offsets || !obj_xy || !out_xy || !out_status)
        return fail(LP2D_ERR_INVALID_ARGUMENT, "NULL data pointer");
    const size_t out_align = (opt.precision == LP2D_PREC_FP64) ? 8 : 4;
    if (!aligned(ax, 4) || !aligned(ay, 4) || !aligned(b, 4) || !aligned(obj_xy, 4) || !aligned(offsets, 8) ||
        !aligned(out_xy, out_align) || !aligned(out_status, 4) || (opt.out_nviol && !aligned(opt.out_nviol, 4)) ||
        (opt.out_def && !aligned(opt.out_def, 4)))
        return fail(LP2D_ERR_INVALID_ARGUMENT, "misaligned pointer");

    const size_t need = lp2d_workspace_bytes(n_lp, &opt);
    const bool ws_usable = workspace && workspace_bytes >= need && aligned(workspace, 8);
    if (opt.schedule == LP2D_SCHED_PERSISTENT) {
        if (!workspace) return fail(LP2D_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", need);
        if (workspace_bytes < need)
            return fail(LP2D_ERR_WORKSPACE, "workspace has %zu bytes, need %zu", workspace_bytes, need);
        if (!aligned(workspace, 8)) return fail(LP2D_ERR_WORKSPACE, "workspace must be 8-byte aligned");
    }

    lp2d::Params p{};
    p.ax = ax;
    p.ay = ay;
    p.b = b;
    p.offsets = offsets;
    p.n_lp = n_lp;
    p.obj = obj_xy;
    p.xmin = box.xmin;
    p.xmax = box.xmax;
    p.ymin = box.ymin;
    p.ymax = box.ymax;
    p.seed = opt.seed;
    p.out_xy = out_xy;
    p.out_status = out_status;
    p.out_nviol = opt.out_nviol;
    p.out_def = opt.out_def;
    // The uniform schedule needs no queue; it records device errors only when given
    // a full-size workspace.
    p.ws = ws_usable ? reinterpret_cast<unsigned long long*>(workspace) : nullptr;
    p.eps32 = opt.eps > 0.0f ? opt.eps : 1e-6f;
    p.eps64 = opt.eps > 0.0f ? static_cast<double>(opt.eps) : 1e-12;
    p.tau = opt.near_parallel_tau > 0.0f ? opt.near_parallel_tau : 1e-3f;
    p.chunk_big = opt.chunk_big > 0 ? (opt.chunk_big < lp2d::kMaxChunk ? opt.chunk_big : lp2d::kMaxChunk)
                                    : lp2d::kDefaultChunkBig;
    p.chunk_small = opt.chunk_small > 0
                        ? (opt.chunk_small < lp2d::kMaxChunkSmall ? opt.chunk_small : lp2d::kMaxChunkSmall)
                        : lp2d::kDefaultChunkSmall;
    p.check_finite = opt.check_finite ? 1 : 0;
    p.team_min = opt.team_min_slots > 0 ? opt.team_min_slots : lp2d::kDefaultTeamMin;
    p.prefetch = opt.l2_prefetch > 0 ? 1 : 0;
    p.lane_max_m = opt.lane_max_m > 0 ? opt.lane_max_m : (opt.lane_max_m == 0 ? lp2d::kDefaultLaneMax : 0);

    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool fp64 = opt.precision == LP2D_PREC_FP64;
    cudaError_t e;
    if (opt.schedule == LP2D_SCHED_UNIFORM) {
        e = fp64 ? lp2d::launch_uniform_f64(p, s) : lp2d::launch_uniform_f32(p, s);
    } else {
        DeviceInfo info;
        int rc = device_info(&info);
        if (rc != LP2D_OK) return rc;
        const int occ = info.occ[opt.precision];
        const int per_sm = opt.ctas_per_sm > 0 ? (opt.ctas_per_sm < occ ? opt.ctas_per_sm : occ) : occ;
        long long grid = static_cast<long long>(info.sms) * per_sm;
        const long long useful = (n_lp + lp2d::kPersistentWarps - 1) / lp2d::kPersistentWarps;
        if (grid > useful) grid = useful;
        if (grid < 1) grid = 1;
        if (fp64) e = lp2d::launch_persistent_f64(p, static_cast<int>(grid), s);
        else if (opt.precision == LP2D_PREC_FP32_F64ISECT) e = lp2d::launch_persistent_mixed(p, static_cast<int>(grid), s);
        else e = lp2d::launch_persistent_f32(p, static_cast<int>(grid), s);
    }
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return ok();
}

int lp2d_solve_batch(const float* ax, const float* ay, const float* b, const int64_t* offsets,
                     int64_t n_lp, const float* obj_xy, lp2d_box box, float* out_xy,
                     int32_t* out_status, lp2d_stream_t stream) {
    if (n_lp <= 0)
        return lp2d_solve_batch_ex(ax, ay, b, offsets, n_lp, obj_xy, box, out_xy, out_status, nullptr, nullptr, 0,
                                   stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = lp2d_workspace_bytes(n_lp, nullptr);
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto key = std::make_pair(dev, s);
        auto it = g_stream_ws.find(key);
        if (it != g_stream_ws.end()) {
            ws = it->second;
        } else {
            e = cudaMalloc(&ws, bytes);
            if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "workspace cudaMalloc: %s", cudaGetErrorString(e));
            e = cudaMemsetAsync(ws, 0, bytes, s);
            if (e != cudaSuccess) {
                cudaFree(ws);
                return fail(LP2D_ERR_CUDA, "workspace memset: %s", cudaGetErrorString(e));
            }
            g_stream_ws[key] = ws;
        }
    }
    return lp2d_solve_batch_ex(ax, ay, b, offsets, n_lp, obj_xy, box, out_xy, out_status, nullptr, ws, bytes, stream);
}

int lp2d_autotune(const float* ax, const float* ay, const float* b, const int64_t* offsets, int64_t n_lp,
                  const float* obj_xy, lp2d_box box, void* out_xy, int32_t* out_status, lp2d_options* opt,
                  void* workspace, size_t workspace_bytes, int reps, float* out_best_ms, lp2d_stream_t stream) {
    if (!opt) return fail(LP2D_ERR_INVALID_ARGUMENT, "opt is NULL (it carries the base options and the result)");
    if (reps < 1) return fail(LP2D_ERR_INVALID_ARGUMENT, "reps = %d < 1", reps);
    if (opt->schedule != LP2D_SCHED_PERSISTENT)
        return fail(LP2D_ERR_UNSUPPORTED, "only the persistent schedule has tuning parameters");
    lp2d_options base = *opt;
    base.out_nviol = nullptr;  // the trial solves write only out_xy / out_status
    base.out_def = nullptr;
    int rc = lp2d_solve_batch_ex(ax, ay, b, offsets, n_lp, obj_xy, box, out_xy, out_status, &base, workspace,
                                 workspace_bytes, stream);  // validates everything once
    if (rc != LP2D_OK) return rc;
    if (n_lp == 0) return ok();
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "events: %s", cudaGetErrorString(e));
    DeviceInfo info;
    rc = device_info(&info);
    if (rc != LP2D_OK) return rc;
    const int occ = info.occ[base.precision];
    const int ctas[2] = {occ, occ > 1 ? occ - 1 : occ};
    const int bigs[3] = {1, 2, 4};
    const int smalls[4] = {1, 2, 4, 8};
    // threads per 1-D LP of a CTA-staged LP: from 512 (or 1024) earlier constraints on
    // the CTA's 128 threads, or always the driving warp's 32 (4096 exceeds every stage)
    const int teams[3] = {512, 1024, 4096};
    // threads per LP: 1 (32 LPs per warp) up to this size, 32 above; -1: always 32
    const int lanes[3] = {-1, 8, lp2d::kCapLane};
    float best = -1.0f;
    lp2d_options winner = base;
    for (int ci = 0; ci < 2 && rc == LP2D_OK; ++ci) {
        if (ci == 1 && ctas[1] == ctas[0]) break;
        for (int bi = 0; bi < 3 && rc == LP2D_OK; ++bi) {
            for (int si = 0; si < 4 * 3 * 3 && rc == LP2D_OK; ++si) {
                lp2d_options o = base;
                o.ctas_per_sm = ctas[ci];
                o.chunk_big = bigs[bi];
                o.chunk_small = smalls[si % 4];
                o.team_min_slots = teams[(si / 4) % 3];
                o.lane_max_m = lanes[si / 12];
                rc = lp2d_solve_batch_ex(ax, ay, b, offsets, n_lp, obj_xy, box, out_xy, out_status, &o, workspace,
                                         workspace_bytes, stream);  // warm-up
                if (rc != LP2D_OK) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && rc == LP2D_OK; ++r)
                    rc = lp2d_solve_batch_ex(ax, ay, b, offsets, n_lp, obj_xy, box, out_xy, out_status, &o,
                                             workspace, workspace_bytes, stream);
                cudaEventRecord(e1, s);
                if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                    rc = fail(LP2D_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= static_cast<float>(reps);
                if (best < 0.0f || ms < best) {
                    best = ms;
                    winner = o;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LP2D_OK) return rc;
    opt->ctas_per_sm = winner.ctas_per_sm;
    opt->chunk_big = winner.chunk_big;
    opt->chunk_small = winner.chunk_small;
    opt->team_min_slots = winner.team_min_slots;
    opt->lane_max_m = winner.lane_max_m;
    if (out_best_ms) *out_best_ms = best;
    return ok();
}

int lp2d_visit_order(uint64_t seed_l, int64_t m, int64_t* out, lp2d_stream_t stream) {
    if (m < 0 || m > (1ll << 26)) return fail(LP2D_ERR_INVALID_ARGUMENT, "m = %lld out of range [0, 2^26]", (long long)m);
    if (m == 0) return ok();
    if (!out || !aligned(out, 8)) return fail(LP2D_ERR_INVALID_ARGUMENT, "out must be a non-NULL int64 pointer");
    cudaError_t e = lp2d::launch_visit_order(seed_l, m, out, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "visit order launch: %s", cudaGetErrorString(e));
    return ok();
}

int lp2d_read_device_error(void* workspace, lp2d_stream_t stream, uint32_t* out_bits) {
    if (!workspace || !out_bits) return fail(LP2D_ERR_INVALID_ARGUMENT, "NULL argument");
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* word = reinterpret_cast<unsigned long long*>(workspace) + lp2d::kWsError;
    unsigned long long host = 0;
    cudaError_t e = cudaMemcpyAsync(&host, word, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(word, 0, sizeof(host), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "reading the error word: %s", cudaGetErrorString(e));
    *out_bits = static_cast<uint32_t>(host);
    return ok();
}

namespace {

// Library-owned pipeline for lp2d_solve_batch_host, one per (device, caller stream):
// two device slots (workspace, inputs and outputs of one chunk each), a stream for the
// host-to-device copies and the events that order them against the solves, which run
// with their device-to-host copies on the caller's stream.
struct HostPipe {
    std::mutex mu;  // held for a whole call: calls on one (device, stream) run one at a time
    char* dev = nullptr;
    size_t slot_bytes = 0;
    cudaStream_t copy = nullptr;
    cudaEvent_t in_ready[2] = {nullptr, nullptr};
    cudaEvent_t solved[2] = {nullptr, nullptr};
    cudaEvent_t entry = nullptr;  // the caller stream at the start of a call
};

std::map<std::pair<int, cudaStream_t>, HostPipe> g_pipes;

size_t up256(size_t n) { return (n + 255) / 256 * 256; }

// Bytes of one slot holding the workspace and up to c constraints and n LPs.
size_t slot_bytes(int64_t c, int64_t n, size_t out_elem) {
    return up256(4 * c) * 3 + up256(8 * (n + 1)) + up256(8 * n) + up256(2 * out_elem * n) + up256(4 * n) +
           up256(sizeof(unsigned long long) * lp2d::kWsWords);
}

}  // namespace

int lp2d_solve_batch_host(const float* ax, const float* ay, const float* b, const int64_t* offsets, int64_t n_lp,
                          const float* obj_xy, lp2d_box box, void* out_xy, int32_t* out_status,
                          const lp2d_options* opt_in, lp2d_stream_t stream) {
    lp2d_options opt;
    if (opt_in) opt = *opt_in;
    else lp2d_default_options(&opt);
    if (opt.out_nviol || opt.out_def)
        return fail(LP2D_ERR_UNSUPPORTED, "out_nviol / out_def are device outputs; use lp2d_solve_batch_ex");
    // options, box and n_lp are checked as for a device call, before anything is enqueued
    lp2d_options ocheck = opt;
    int rc0 = lp2d_solve_batch_ex(nullptr, nullptr, nullptr, nullptr, n_lp < 0 ? n_lp : 0, nullptr, box, nullptr,
                                  nullptr, &ocheck, nullptr, 0, stream);
    if (rc0 != LP2D_OK) return rc0;
    if (n_lp == 0) return ok();
    if (!ax || !ay || !b || !offsets || !obj_xy || !out_xy || !out_status)
        return fail(LP2D_ERR_INVALID_ARGUMENT, "NULL host pointer");
    for (int64_t l = 0; l < n_lp; ++l)
        if (offsets[l + 1] < offsets[l])
            return fail(LP2D_ERR_INVALID_ARGUMENT, "offsets decrease at LP %lld", (long long)l);
    if (offsets[0] < 0) return fail(LP2D_ERR_INVALID_ARGUMENT, "offsets[0] < 0");
    const size_t out_elem = (opt.precision == LP2D_PREC_FP64) ? 8 : 4;
    const int64_t total = offsets[n_lp] - offsets[0];

    // Chunk plan, cut at LP boundaries.  Copies run at the host link's rate and the
    // solve of a chunk takes about a quarter of its copy time, so the call costs about
    // the copy of the whole batch plus the solve of the last chunk: chunks shrink
    // towards the end (40/30/17/9/4 % of the last 160M constraints), and anything
    // before that goes in equal chunks of at most 64M constraints to bound the slots.
    // Every split of a copy costs some link throughput, so small batches stay whole.
    std::vector<int64_t> targets;  // constraint counts from offsets[0] at the cuts
    constexpr int64_t kWholeBelow = 2 << 20, kTail = 160ll << 20, kHeadChunk = 64ll << 20;
    if (total >= kWholeBelow) {
        const int64_t head = total > kTail ? total - kTail : 0;
        const int64_t nh = (head + kHeadChunk - 1) / kHeadChunk;
        for (int64_t i = 1; i <= nh; ++i) targets.push_back(head * i / nh);
        static const int kTailPermille[4] = {400, 700, 870, 960};
        for (int i = 0; i < 4; ++i) targets.push_back(head + (total - head) * kTailPermille[i] / 1000);
    }
    std::vector<int64_t> cut;
    cut.push_back(0);
    for (int64_t t : targets) {
        int64_t c = std::lower_bound(offsets, offsets + n_lp + 1, offsets[0] + t) - offsets;
        if (c > n_lp) c = n_lp;
        if (c > cut.back()) cut.push_back(c);
    }
    if (cut.back() < n_lp) cut.push_back(n_lp);
    const int64_t k = static_cast<int64_t>(cut.size()) - 1;
    int64_t max_c = 0, max_n = 0;
    for (int64_t i = 0; i < k; ++i) {
        max_c = std::max(max_c, offsets[cut[i + 1]] - offsets[cut[i]]);
        max_n = std::max(max_n, cut[i + 1] - cut[i]);
    }
    const size_t need = slot_bytes(max_c, max_n, out_elem);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    const cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    HostPipe* pp = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);  // map nodes stay where they are once inserted
        pp = &g_pipes[std::make_pair(dev, cs)];
    }
    HostPipe& p = *pp;
    std::lock_guard<std::mutex> pipe_lock(p.mu);
    {
        if (!p.copy) {
            if ((e = cudaStreamCreateWithFlags(&p.copy, cudaStreamNonBlocking)) != cudaSuccess)
                return fail(LP2D_ERR_CUDA, "copy stream: %s", cudaGetErrorString(e));
            for (int i = 0; i < 2; ++i) {
                cudaEventCreateWithFlags(&p.in_ready[i], cudaEventDisableTiming);
                cudaEventCreateWithFlags(&p.solved[i], cudaEventDisableTiming);
            }
            cudaEventCreateWithFlags(&p.entry, cudaEventDisableTiming);
        }
        if (p.slot_bytes < need) {
            // earlier work of this pipeline may still use the old slots
            if (p.dev) {
                cudaStreamSynchronize(p.copy);
                cudaStreamSynchronize(cs);
                cudaFree(p.dev);
                p.dev = nullptr;
                p.slot_bytes = 0;
            }
            if ((e = cudaMalloc(&p.dev, 2 * need)) != cudaSuccess)
                return fail(LP2D_ERR_CUDA, "pipeline buffers (%zu bytes): %s", 2 * need, cudaGetErrorString(e));
            if ((e = cudaMemset(p.dev, 0, 2 * need)) != cudaSuccess)  // zeroed workspaces
                return fail(LP2D_ERR_CUDA, "pipeline memset: %s", cudaGetErrorString(e));
            p.slot_bytes = need;
        }
    }
    // copies of a call start after the caller's earlier work on its stream
    if ((e = cudaEventRecord(p.entry, cs)) != cudaSuccess || (e = cudaStreamWaitEvent(p.copy, p.entry, 0)) != cudaSuccess)
        return fail(LP2D_ERR_CUDA, "ordering: %s", cudaGetErrorString(e));
    for (int64_t i = 0; i < k; ++i) {
        const int s = static_cast<int>(i & 1);
        const int64_t lo = cut[i], hi = cut[i + 1], n = hi - lo;
        if (n == 0) continue;
        const int64_t c0 = offsets[lo], c = offsets[hi] - c0;
        // the workspace sits at the start of the slot, at the same place for every call
        char* dws = p.dev + s * p.slot_bytes;
        char* base = dws + up256(sizeof(unsigned long long) * lp2d::kWsWords);
        float* dax = reinterpret_cast<float*>(base);
        float* day = reinterpret_cast<float*>(base + up256(4 * max_c));
        float* db = reinterpret_cast<float*>(base + 2 * up256(4 * max_c));
        int64_t* doff = reinterpret_cast<int64_t*>(base + 3 * up256(4 * max_c));
        float* dobj = reinterpret_cast<float*>(reinterpret_cast<char*>(doff) + up256(8 * (max_n + 1)));
        char* dxy = reinterpret_cast<char*>(dobj) + up256(8 * max_n);
        int32_t* dst = reinterpret_cast<int32_t*>(dxy + up256(2 * out_elem * max_n));
        // slot s is free once the solve and copy-out of chunk i-2 are done
        if (i >= 2 && (e = cudaStreamWaitEvent(p.copy, p.solved[s], 0)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(dax, ax + c0, 4 * c, cudaMemcpyHostToDevice, p.copy)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(day, ay + c0, 4 * c, cudaMemcpyHostToDevice, p.copy)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(db, b + c0, 4 * c, cudaMemcpyHostToDevice, p.copy)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(doff, offsets + lo, 8 * (n + 1), cudaMemcpyHostToDevice, p.copy)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(dobj, obj_xy + 2 * lo, 8 * n, cudaMemcpyHostToDevice, p.copy)) != cudaSuccess) break;
        if ((e = cudaEventRecord(p.in_ready[s], p.copy)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(cs, p.in_ready[s], 0)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(dws, 0, sizeof(unsigned long long) * lp2d::kWsWords, cs)) != cudaSuccess) break;
        // offsets stay absolute: the constraint arrays are passed shifted back by c0
        // element addresses (in integer arithmetic: the shifted address lies outside the
        // slot, and the kernels only ever add offsets >= c0 to it)
        lp2d_options oc = opt;
        oc.seed = opt.seed + static_cast<uint64_t>(lo);
        auto back = [c0](const float* q) {
            return reinterpret_cast<const float*>(reinterpret_cast<uintptr_t>(q) -
                                                  static_cast<uintptr_t>(c0) * sizeof(float));
        };
        const int rc = lp2d_solve_batch_ex(back(dax), back(day), back(db), doff, n, dobj, box, dxy, dst, &oc, dws,
                                           up256(sizeof(unsigned long long) * lp2d::kWsWords), stream);
        if (rc != LP2D_OK) return rc;
        // results (12 bytes per LP) go back on the solve stream, so the copy stream never
        // waits for a solve except to reuse a slot
        if ((e = cudaMemcpyAsync(static_cast<char*>(out_xy) + 2 * out_elem * lo, dxy, 2 * out_elem * n,
                                 cudaMemcpyDeviceToHost, cs)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(out_status + lo, dst, 4 * n, cudaMemcpyDeviceToHost, cs)) != cudaSuccess) break;
        if ((e = cudaEventRecord(p.solved[s], cs)) != cudaSuccess) break;
    }
    if (e != cudaSuccess) return fail(LP2D_ERR_CUDA, "host pipeline: %s", cudaGetErrorString(e));
    return ok();
}

const char* lp2d_last_error(void) { return g_last_error; }

const char* lp2d_version(void) { return "lp2d 0.1.0 (sm_103a)"; }

}  // extern "C"
