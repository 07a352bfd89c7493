// lp3d.cu -- the batched 3-D Seidel solver and its extern "C" entry point.
//
// The paper's method one dimension up (Sec. 2.1 gives it in 2-D; Sec. 6 names higher
// dimensions as the next step).  One warp solves one LP staged in shared memory in
// visit order: slots 0..5 hold the box planes (x <= xmax, -x <= -xmin, y <= ymax,
// -y <= -ymin, z <= zmax, -z <= -zmin), slot 6 + p the constraint visited at p.
//   - scan: 32 positions per step against the current optimum; the first violated
//     one is the next step of serial Seidel;
//   - a violation of plane h: the new optimum lies on h.  The plane is written as
//     p0 + s u + t w (p0 = h hb / |h|^2, u = h x e_j with e_j the axis of the smallest
//     |h_j|, w = h x u) and the 2-D LP on it runs over the box and every earlier
//     constraint, projected on the fly: it starts at the best of the fifteen
//     intersections of pairs of box planes (one per lane) and is itself Seidel's
//     2-D method, whose violations solve 1-D LPs on lines (Eqs. 3, 4) with the
//     2-D solver's rules (lanes reduce strided slots, redux.sync combines them);
//   - an infeasible 2-D LP makes the LP infeasible.
// A persistent grid of 4-warp CTAs pulls LPs from two queues: LPs of 507..1018
// constraints go to warps 0 and 1 with half of the CTA's stage each, smaller ones to
// all four warps with a quarter each.  A second, one-warp-per-CTA kernel launched
// after it takes the LPs of 1019..12282 constraints from a third queue, each staged
// in about 200 KB of dynamic shared memory; larger LPs are reported as BAD_INPUT.
#include <cstdarg>
#include <cstdio>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <set>
#include <utility>

#include "lp3d.h"
#include "lp2d_internal.h"
#include "lp2d_staged.cuh"
#include "lp_stage_big.cuh"

namespace lp2d {

constexpr int kBox3 = 6;
constexpr int kQuarter3 = 512;  // stage slots of a warp in the small-LP phase
constexpr int kHalf3 = 1024;    // stage slots of a warp in the mid-size phase
constexpr int kCap3Small = kQuarter3 - kBox3;
constexpr int kCap3Mid = kHalf3 - kBox3;
constexpr int kStage3 = 4 * kQuarter3;
constexpr int kWarps3 = 4;
constexpr unsigned kDevErrTooLarge = 4u;
// The large-LP kernel: one warp per CTA, a stage of kStage3L slots per array and a key
// bitmap for domains up to 4^7 = 16384 bits, in dynamic shared memory.
constexpr int kStage3L = 12288;
constexpr int kCap3Large = kStage3L - kBox3;
constexpr int kWords3L = 512;
constexpr size_t kSmem3L = sizeof(float) * 4 * kStage3L + sizeof(unsigned) * kWords3L + sizeof(int) * kWords3L;
constexpr int kWsDoneLarge = 5;  // workspace word: large-LP CTAs that have finished

struct Params3 {
    const float* __restrict__ ax;
    const float* __restrict__ ay;
    const float* __restrict__ az;
    const float* __restrict__ b;
    const int64_t* __restrict__ offsets;
    int64_t n_lp;
    const float* __restrict__ obj;
    float box[6];
    uint64_t seed;
    void* out_xyz;
    int32_t* out_status;
    int32_t* out_nviol;
    int32_t* out_def;
    unsigned long long* ws;
    float eps32;
    double eps64;
    int chunk;
    int check_finite;
    // least-violation mode: LPs whose status_in is INFEASIBLE, read from 2-D arrays
    // (az = -|(ax, ay)|, objective (0, 0, -1)); x, y go to out_xyz with a stride of 2
    // and the violation to out_t
    const int32_t* __restrict__ status_in;
    float* out_t;
};

template <typename Real>
__device__ __forceinline__ bool violates3(Real gx, Real gy, Real gz, Real gb, Real x, Real y, Real z, Real eps) {
    const Real s = gx * x + gy * y + gz * z - gb;
    const Real tol = eps * (real_abs(gx * x) + real_abs(gy * y) + real_abs(gz * z) + real_abs(gb));
    return s > tol;
}

__device__ __forceinline__ void write_box3(const Params3& P, float* sX, float* sY, float* sZ, float* sB, int lane) {
    if (lane < kBox3) {
        const int axis = lane >> 1;
        const float sg = (lane & 1) ? -1.0f : 1.0f;
        sX[lane] = axis == 0 ? sg : 0.0f;
        sY[lane] = axis == 1 ? sg : 0.0f;
        sZ[lane] = axis == 2 ? sg : 0.0f;
        sB[lane] = (lane & 1) ? -P.box[2 * axis] : P.box[2 * axis + 1];
    }
}

// Warp staging of a 3-D LP with m <= 1018 constraints (key domain <= 1024 bits, one
// bitmap word per lane), as the 2-D warp staging with a fourth array.
__device__ __forceinline__ void stage_lp3_warp(const VisitOrder& vo, int m, const float* __restrict__ gax,
                                               const float* __restrict__ gay, const float* __restrict__ gaz,
                                               const float* __restrict__ gb, float* sX, float* sY, float* sZ,
                                               float* sB, unsigned* bm, int lane) {
    bm[lane] = 0u;
    __syncwarp();
    for (int q = lane; q < m; q += 32) {
        const uint32_t e = vo.enc(static_cast<uint32_t>(q));
        atomicOr(bm + (e >> 5), 1u << (e & 31u));
    }
    __syncwarp();
    const unsigned w = bm[lane];
    const int excl = warp_inclusive_scan(__popc(w), lane) - __popc(w);
    for (int q0 = 0; q0 < m; q0 += 32) {
        const int q = q0 + lane;
        const bool valid = q < m;
        const uint32_t e = vo.enc(static_cast<uint32_t>(valid ? q : 0));
        const int src = static_cast<int>(e >> 5);
        const unsigned we = __shfl_sync(kFull, w, src);
        const int pe = __shfl_sync(kFull, excl, src);
        if (valid) {
            const int slot = kBox3 + pe + __popc(we & ((1u << (e & 31u)) - 1u));
            cp_async4(sX + slot, gax + q);
            cp_async4(sY + slot, gay + q);
            if (gaz) cp_async4(sZ + slot, gaz + q);
            cp_async4(sB + slot, gb + q);
        }
    }
}

// Constraint id of a stage slot for out_def: -1 - plane for the box, otherwise the
// index of the constraint staged there.
__device__ __forceinline__ int slot_id3(int slot, const VisitOrder& vo, const unsigned* bm, int lane) {
    if (slot < kBox3) return -1 - slot;
    const uint64_t dw = vo.domain() >> 5;
    const int nwords = dw > 0 ? static_cast<int>(dw) : 1;
    return static_cast<int>(vo.dec(bitmap_select(bm, nwords, slot - kBox3, lane)));
}

// Seidel's method on one staged 3-D LP by one warp; writes the LP's outputs.
template <typename Real>
__device__ void drive_lp3(const Params3& P, int64_t lp, int m, const VisitOrder& vo, const float* __restrict__ sX,
                          const float* __restrict__ sY, const float* __restrict__ sZ, const float* __restrict__ sB,
                          const unsigned* bm, int lane) {
    using KT = KeyOf<Real>;
    using K = typename KT::type;
    const bool fallback = P.status_in != nullptr;
    const float cxf = fallback ? 0.0f : __ldg(P.obj + 3 * lp), cyf = fallback ? 0.0f : __ldg(P.obj + 3 * lp + 1);
    const float czf = fallback ? -1.0f : __ldg(P.obj + 3 * lp + 2);
    const Real cx = cxf, cy = cyf, cz = czf;
    const Real eps = (sizeof(Real) == 4) ? Real(P.eps32) : Real(P.eps64);
    Real vx = cx >= Real(0) ? Real(P.box[1]) : Real(P.box[0]);
    Real vy = cy >= Real(0) ? Real(P.box[3]) : Real(P.box[2]);
    Real vz = cz >= Real(0) ? Real(P.box[5]) : Real(P.box[4]);
    int d0 = cx >= Real(0) ? 0 : 1, d1 = cy >= Real(0) ? 2 : 3, d2 = cz >= Real(0) ? 4 : 5;
    int status = -1, nviol = 0;
    float fin = 0.0f;
    int k = 0;
    while (k < m) {
        const int p = k + lane;
        bool viol = false;
        if (p < m) {
            const int sl = kBox3 + p;
            const float fx = sX[sl], fy = sY[sl], fz = sZ[sl], fb = sB[sl];
            fin = fmaf(fx, 0.0f, fmaf(fy, 0.0f, fmaf(fz, 0.0f, fmaf(fb, 0.0f, fin))));
            viol = violates3<Real>(fx, fy, fz, fb, vx, vy, vz, eps);
        }
        const unsigned bal = __ballot_sync(kFull, viol);
        if (bal == 0u) {
            k += 32;
            continue;
        }
        const int first = k + __ffs(bal) - 1;
        const int fslot = kBox3 + first;
        k = first + 1;
        // ---- the violated plane h.x = hb
        const Real hx = sX[fslot], hy = sY[fslot], hz = sZ[fslot], hb = sB[fslot];
        const Real n2 = hx * hx + hy * hy + hz * hz;
        if (!(n2 != Real(0))) {  // 0.x <= hb < 0 (NaN data also stops here)
            status = kInfeasible;
            break;
        }
        const Real sc = hb / n2;
        const Real p0x = hx * sc, p0y = hy * sc, p0z = hz * sc;
        int ja = 0;
        if (real_abs(hy) < real_abs(hx)) ja = 1;
        if (real_abs(hz) < (ja == 0 ? real_abs(hx) : real_abs(hy))) ja = 2;
        // u = h x e_ja, w = h x u
        const Real ux = ja == 0 ? Real(0) : (ja == 1 ? -hz : hy);
        const Real uy = ja == 0 ? hz : (ja == 1 ? Real(0) : -hx);
        const Real uz = ja == 0 ? -hy : (ja == 1 ? hx : Real(0));
        const Real wx = hy * uz - hz * uy, wy = hz * ux - hx * uz, wz = hx * uy - hy * ux;
        const Real cs = cx * ux + cy * uy + cz * uz, ct = cx * wx + cy * wy + cz * wz;
        ++nviol;
        // ---- start of the 2-D LP: the best intersection of two box planes (lane = pair)
        bool ok = false;
        Real ss = Real(0), tt = Real(0), val = Real(0);
        int pi = 0, pj = 0;
        if (lane < 15) {
            // pairs (i, j), i < j, in order: lane -> (i, j)
            pi = lane < 5 ? 0 : lane < 9 ? 1 : lane < 12 ? 2 : lane < 14 ? 3 : 4;
            const int before = pi == 0 ? 0 : pi == 1 ? 5 : pi == 2 ? 9 : pi == 3 ? 12 : 14;
            pj = pi + 1 + (lane - before);
            const Real gix = sX[pi], giy = sY[pi], giz = sZ[pi], gib = sB[pi];
            const Real gjx = sX[pj], gjy = sY[pj], gjz = sZ[pj], gjb = sB[pj];
            const Real bsi = gix * ux + giy * uy + giz * uz, bti = gix * wx + giy * wy + giz * wz;
            const Real bri = gib - (gix * p0x + giy * p0y + giz * p0z);
            const Real bsj = gjx * ux + gjy * uy + gjz * uz, btj = gjx * wx + gjy * wy + gjz * wz;
            const Real brj = gjb - (gjx * p0x + gjy * p0y + gjz * p0z);
            const Real det = bsi * btj - bti * bsj;
            if (det != Real(0)) {
                ss = (bri * btj - bti * brj) / det;
                tt = (bsi * brj - bri * bsj) / det;
                const Real X = p0x + ss * ux + tt * wx, Y = p0y + ss * uy + tt * wy, Z = p0z + ss * uz + tt * wz;
                ok = true;
#pragma unroll
                for (int f = 0; f < kBox3; ++f)
                    if (f != pi && f != pj && violates3<Real>(sX[f], sY[f], sZ[f], sB[f], X, Y, Z, eps)) ok = false;
                val = cs * ss + ct * tt;
            }
        }
        const unsigned okb = __ballot_sync(kFull, ok);
        bool infeasible2 = okb == 0u;  // the plane misses the box
        Real s = Real(0), t = Real(0);
        int e0 = kNoPos, e1 = kNoPos;
        if (!infeasible2) {
            K key = ok ? KT::key(val) : KT::key(-real_inf<Real>());
            int who = ok ? lane : kNoPos;
            warp_max_pair(key, who);  // the largest value, the first pair on ties
            s = __shfl_sync(kFull, ss, who);
            t = __shfl_sync(kFull, tt, who);
            e0 = __shfl_sync(kFull, pi, who);
            e1 = __shfl_sync(kFull, pj, who);
            // ---- Seidel's 2-D method on the plane over positions 0..first-1
            int j = 0;
            while (j < first) {
                const Real X = p0x + s * ux + t * wx, Y = p0y + s * uy + t * wy, Z = p0z + s * uz + t * wz;
                const int q = j + lane;
                bool v2 = false;
                if (q < first) {
                    const int sl = kBox3 + q;
                    v2 = violates3<Real>(sX[sl], sY[sl], sZ[sl], sB[sl], X, Y, Z, eps);
                }
                const unsigned b2 = __ballot_sync(kFull, v2);
                if (b2 == 0u) {
                    j += 32;
                    continue;
                }
                const int fj = j + __ffs(b2) - 1;
                const int gslot = kBox3 + fj;
                j = fj + 1;
                const Real gx = sX[gslot], gy = sY[gslot], gz = sZ[gslot], gb = sB[gslot];
                const Real gs = gx * ux + gy * uy + gz * uz, gt = gx * wx + gy * wy + gz * wz;
                const Real gr = gb - (gx * p0x + gy * p0y + gz * p0z);
                const Real nn = gs * gs + gt * gt;
                if (!(nn != Real(0))) {  // g's plane is parallel to h's and excludes all of it
                    infeasible2 = true;
                    break;
                }
                const Real q0s = gs * (gr / nn), q0t = gt * (gr / nn);
                // direction of the line, oriented so that the objective's end is the
                // right end (the left end of (-gt, gs) when they are perpendicular)
                const Real cd = cs * (-gt) + ct * gs;
                const Real fsg = cd > Real(0) ? Real(1) : Real(-1);
                const Real ds = -gt * fsg, dt = gs * fsg;
                Real thi = real_inf<Real>(), tlo = -real_inf<Real>();
                int phi = kNoPos;
                const Real ninf = -real_inf<Real>();
                for (int f = lane; f < gslot; f += 32) {
                    const Real fx = sX[f], fy = sY[f], fz = sZ[f], fb = sB[f];
                    const Real fs = fx * ux + fy * uy + fz * uz, ft = fx * wx + fy * wy + fz * wz;
                    const Real fr = fb - (fx * p0x + fy * p0y + fz * p0z);
                    const Real den = (fs * ds + ft * dt) + Real(0);
                    const Real num = fr - (fs * q0s + ft * q0t);
                    const Real tau = real_div<Real>(num, den);
                    const bool right = den >= Real(0);
                    const bool take = right && (tau < thi);
                    thi = take ? tau : thi;
                    phi = take ? f : phi;
                    tlo = real_max<Real>(tlo, right ? ninf : tau);
                }
                warp_reduce_1dlp<Real>(thi, phi, tlo);
                if (!(tlo <= thi)) {  // empty interval, or a parallel constraint excludes the line
                    infeasible2 = true;
                    break;
                }
                s = q0s + thi * ds;
                t = q0t + thi * dt;
                e0 = gslot;
                e1 = phi;
            }
        }
        if (infeasible2) {
            status = kInfeasible;
            break;
        }
        vx = p0x + s * ux + t * wx;
        vy = p0y + s * uy + t * wy;
        vz = p0z + s * uz + t * wz;
        d0 = fslot;
        d1 = e0;
        d2 = e1;
    }
    if (P.check_finite) {
        for (int p = k + lane; p < m; p += 32)
            fin = fmaf(sX[kBox3 + p], 0.0f,
                       fmaf(sY[kBox3 + p], 0.0f, fmaf(sZ[kBox3 + p], 0.0f, fmaf(sB[kBox3 + p], 0.0f, fin))));
    }
    const bool bad_data = P.check_finite && __any_sync(kFull, fin != fin);
    const bool bad_obj =
        !(fabsf(cxf) <= 3.402823466e38f) || !(fabsf(cyf) <= 3.402823466e38f) || !(fabsf(czf) <= 3.402823466e38f);
    int id0 = 0, id1 = 0, id2 = 0;
    if (P.out_def) {
        id0 = slot_id3(d0, vo, bm, lane);
        id1 = slot_id3(d1, vo, bm, lane);
        id2 = slot_id3(d2, vo, bm, lane);
    }
    if (lane == 0) {
        if (bad_data || bad_obj) status = kBadInput;
        else if (status < 0) status = (d0 < kBox3 || d1 < kBox3 || d2 < kBox3) ? kBoxBounded : kOptimal;
        Real* out = reinterpret_cast<Real*>(P.out_xyz);
        const bool none = status == kInfeasible || status == kBadInput;
        const Real nan = real_inf<Real>() - real_inf<Real>();
        if (fallback) {
            out[2 * lp] = none ? nan : vx;
            out[2 * lp + 1] = none ? nan : vy;
            if (P.out_t) P.out_t[lp] = none ? nan : static_cast<float>(vz);
        } else {
            out[3 * lp] = none ? nan : vx;
            out[3 * lp + 1] = none ? nan : vy;
            out[3 * lp + 2] = none ? nan : vz;
        }
        P.out_status[lp] = status;
        if (P.out_nviol) P.out_nviol[lp] = nviol;
        if (P.out_def) {
            P.out_def[3 * lp] = id0;
            P.out_def[3 * lp + 1] = id1;
            P.out_def[3 * lp + 2] = id2;
        }
    }
}

template <typename Real>
__device__ __forceinline__ void write_bad3(const Params3& P, int64_t lp, unsigned bits) {
    atomicOr(P.ws + kWsError, static_cast<unsigned long long>(bits));
    P.out_status[lp] = kBadInput;
    Real* out = reinterpret_cast<Real*>(P.out_xyz);
    const Real nan = real_inf<Real>() - real_inf<Real>();
    if (P.status_in != nullptr) {
        out[2 * lp] = out[2 * lp + 1] = nan;
        if (P.out_t) P.out_t[lp] = nan;
    } else {
        out[3 * lp] = out[3 * lp + 1] = out[3 * lp + 2] = nan;
    }
}

// One warp's loop over a queue: grab spans of LP indices (doubling after a grab
// without LPs of the class, halving after one with more than the target), stage and
// solve the LPs of size (lo, hi] among them.
template <typename Real, bool kLarge = false>
__device__ void warp_queue3(const Params3& P, unsigned long long* head, long long lo, long long hi, float* sX,
                            float* sY, float* sZ, float* sB, unsigned* bm, int lane, int* pre = nullptr) {
    constexpr long long kCap = kLarge ? kCap3Large : kCap3Mid;
    int span = P.chunk;
    for (;;) {
        long long start = 0;
        if (lane == 0) start = static_cast<long long>(atomicAdd(head, static_cast<unsigned long long>(span)));
        start = __shfl_sync(kFull, start, 0);
        if (start < 0 || start >= P.n_lp) break;  // a head past 2^63 is not a valid LP index
        const bool in = lane < span && start + lane < P.n_lp;
        long long off_l = 0, mm_l = 0;
        if (in) {
            off_l = __ldg(P.offsets + start + lane);
            mm_l = __ldg(P.offsets + start + lane + 1) - off_l;
        }
        const bool wanted = P.status_in == nullptr || (in && __ldg(P.status_in + start + lane) == kInfeasible);
        unsigned todo = __ballot_sync(kFull, in && wanted && mm_l > lo && mm_l <= hi);
        const int found = __popc(todo);
        span = found == 0 ? min(2 * span, 32) : (found > P.chunk ? max(span >> 1, 1) : span);
        while (todo != 0u) {
            const int i = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int64_t lp = start + i;
            const long long base = __shfl_sync(kFull, off_l, i);
            const long long mm = __shfl_sync(kFull, mm_l, i);
            if (mm < 0 || mm > kCap) {
                if (lane == 0) write_bad3<Real>(P, lp, mm < 0 ? kDevErrBadOffsets : kDevErrTooLarge);
                continue;
            }
            const int m = static_cast<int>(mm);
            VisitOrder vo;
            warp_visit_order(vo, P.seed + static_cast<uint64_t>(lp), static_cast<uint32_t>(m), lane);
            write_box3(P, sX, sY, sZ, sB, lane);
            if constexpr (kLarge) {
                const float* gax = P.ax + base;
                const float* gay = P.ay + base;
                const float* gaz = P.az ? P.az + base : nullptr;
                const float* gb = P.b + base;
                stage_ranks_warp(vo, m, bm, pre, lane, [&](int r, int q) {
                    const int slot = kBox3 + r;
                    cp_async4(sX + slot, gax + q);
                    cp_async4(sY + slot, gay + q);
                    if (gaz) cp_async4(sZ + slot, gaz + q);
                    cp_async4(sB + slot, gb + q);
                });
            } else {
                stage_lp3_warp(vo, m, P.ax + base, P.ay + base, P.az ? P.az + base : nullptr, P.b + base, sX, sY,
                               sZ, sB, bm, lane);
            }
            cp_async_wait_all();
            __syncwarp();
            if (P.az == nullptr) {
                // least violation: the third coefficient is -|(ax, ay)| (each product and
                // the sum rounded separately, so that it equals the plain float32 value)
                for (int i = lane; i < m; i += 32) {
                    const int sl = kBox3 + i;
                    sZ[sl] = -sqrtf(__fadd_rn(__fmul_rn(sX[sl], sX[sl]), __fmul_rn(sY[sl], sY[sl])));
                }
                __syncwarp();
            }
            drive_lp3<Real>(P, lp, m, vo, sX, sY, sZ, sB, bm, lane);
            __syncwarp();  // all lanes are done with the stage before it is overwritten
        }
    }
}

// FP32: fitted to 6 resident CTAs per SM (the limit of its shared memory).
template <typename Real>
__global__ void __launch_bounds__(kWarps3 * 32, sizeof(Real) == 4 ? 6 : 1) seidel3_kernel(const Params3 P) {
    __shared__ float sX[kStage3];
    __shared__ float sY[kStage3];
    __shared__ float sZ[kStage3];
    __shared__ float sB[kStage3];
    __shared__ unsigned s_bm[kWarps3 * 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned long long* ws = P.ws;
    // mid-size LPs: warps 0 and 1, half a stage each
    if (warp < 2)
        warp_queue3<Real>(P, ws + kWsHeadMid, kCap3Small, kCap3Mid, sX + warp * kHalf3, sY + warp * kHalf3,
                          sZ + warp * kHalf3, sB + warp * kHalf3, s_bm + warp * 32, lane);
    __syncthreads();
    // small LPs (and negative sizes): every warp, a quarter of the stage each
    warp_queue3<Real>(P, ws + kWsHeadSmall, -(1ll << 62), kCap3Small, sX + warp * kQuarter3, sY + warp * kQuarter3,
                      sZ + warp * kQuarter3, sB + warp * kQuarter3, s_bm + warp * 32, lane);
    // the last CTA out resets the queue heads for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(ws + kWsDone, 1ull);
        if (prev == static_cast<unsigned long long>(gridDim.x) - 1ull) {
            atomicExch(ws + kWsHeadMid, 0ull);
            atomicExch(ws + kWsHeadSmall, 0ull);
            atomicExch(ws + kWsDone, 0ull);
        }
    }
}

// LPs above kCap3Mid constraints: one warp per CTA with a stage of kStage3L slots;
// LPs above kCap3Large are reported as too large.  Runs after seidel3_kernel on the
// same stream, with its own queue head and done counter.
template <typename Real>
__global__ void __launch_bounds__(32, 1) seidel3_large_kernel(const Params3 P) {
    extern __shared__ __align__(16) unsigned char smem3l[];
    float* sX = reinterpret_cast<float*>(smem3l);
    float* sY = sX + kStage3L;
    float* sZ = sY + kStage3L;
    float* sB = sZ + kStage3L;
    unsigned* bm = reinterpret_cast<unsigned*>(sB + kStage3L);
    int* pre = reinterpret_cast<int*>(bm + kWords3L);
    const int lane = threadIdx.x;
    unsigned long long* ws = P.ws;
    warp_queue3<Real, true>(P, ws + kWsHeadBig, kCap3Mid, 1ll << 62, sX, sY, sZ, sB, bm, lane, pre);
    if (lane == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(ws + kWsDoneLarge, 1ull);
        if (prev == static_cast<unsigned long long>(gridDim.x) - 1ull) {
            atomicExch(ws + kWsHeadBig, 0ull);
            atomicExch(ws + kWsDoneLarge, 0ull);
        }
    }
}

}  // namespace lp2d

namespace {

bool aligned3(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int occupancy3(bool fp64, int* sms, int* per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, lp2d::seidel3_kernel<double>,
                                                                 lp2d::kWarps3 * 32, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, lp2d::seidel3_kernel<float>,
                                                                 lp2d::kWarps3 * 32, 0);
    if (e != cudaSuccess) return lp2d::report_error(LP2D_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    if (*per_sm < 1) return lp2d::report_error(LP2D_ERR_CUDA, "3-D kernel cannot be resident");
    return LP2D_OK;
}

}  // namespace

namespace {

// Opt the large-LP kernel in to its dynamic shared memory, once per device and precision.
std::mutex g_large3_mu;
std::set<std::pair<int, bool>> g_large3_ready;

int large3_ready(bool fp64) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lp2d::report_error(LP2D_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_large3_mu);
    if (g_large3_ready.count({dev, fp64})) return LP2D_OK;
    e = fp64 ? cudaFuncSetAttribute(lp2d::seidel3_large_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(lp2d::kSmem3L))
             : cudaFuncSetAttribute(lp2d::seidel3_large_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(lp2d::kSmem3L));
    if (e != cudaSuccess)
        return lp2d::report_error(LP2D_ERR_CUDA, "large-LP kernel shared memory: %s", cudaGetErrorString(e));
    g_large3_ready.insert({dev, fp64});
    return LP2D_OK;
}

int launch3(lp2d::Params3& p, const lp2d_options& opt, int64_t n_lp, lp2d_stream_t stream) {
    using lp2d::report_error;
    const bool fp64 = opt.precision == LP2D_PREC_FP64;
    int sms = 0, per_sm = 0;
    int rc = occupancy3(fp64, &sms, &per_sm);
    if (rc != LP2D_OK) return rc;
    if (opt.ctas_per_sm > 0 && opt.ctas_per_sm < per_sm) per_sm = opt.ctas_per_sm;
    long long grid = static_cast<long long>(sms) * per_sm;
    const long long useful = (n_lp + lp2d::kWarps3 - 1) / lp2d::kWarps3;
    if (grid > useful) grid = useful;
    if (grid < 1) grid = 1;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (fp64) lp2d::seidel3_kernel<double><<<static_cast<int>(grid), lp2d::kWarps3 * 32, 0, s>>>(p);
    else lp2d::seidel3_kernel<float><<<static_cast<int>(grid), lp2d::kWarps3 * 32, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(LP2D_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    // LPs above the stage of a warp pair: one CTA per SM, each a warp with ~200 KB
    rc = large3_ready(fp64);
    if (rc != LP2D_OK) return rc;
    const int lgrid = static_cast<int>(std::min<long long>(sms, n_lp));
    if (fp64) lp2d::seidel3_large_kernel<double><<<lgrid, 32, lp2d::kSmem3L, s>>>(p);
    else lp2d::seidel3_large_kernel<float><<<lgrid, 32, lp2d::kSmem3L, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(LP2D_ERR_CUDA, "large-LP kernel launch: %s", cudaGetErrorString(e));
    return LP2D_OK;
}

int check_options3(const lp2d_options& opt) {
    using lp2d::report_error;
    if (opt.precision != LP2D_PREC_FP32 && opt.precision != LP2D_PREC_FP64)
        return report_error(LP2D_ERR_UNSUPPORTED, "the 3-D solver runs in FP32 or FP64");
    if (opt.schedule != LP2D_SCHED_PERSISTENT)
        return report_error(LP2D_ERR_UNSUPPORTED, "the 3-D solver has the persistent schedule only");
    if (opt.chunk_small < 0 || !(opt.eps >= 0.0f) || !std::isfinite(opt.eps))
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "bad tuning parameter or eps");
    return LP2D_OK;
}

void fill_common3(lp2d::Params3& p, const lp2d_options& opt, void* workspace) {
    p.seed = opt.seed;
    p.out_nviol = opt.out_nviol;
    p.out_def = opt.out_def;
    p.ws = reinterpret_cast<unsigned long long*>(workspace);
    p.eps32 = opt.eps > 0.0f ? opt.eps : 1e-6f;
    p.eps64 = opt.eps > 0.0f ? static_cast<double>(opt.eps) : 1e-12;
    p.chunk = opt.chunk_small > 0 ? (opt.chunk_small < lp2d::kMaxChunkSmall ? opt.chunk_small : lp2d::kMaxChunkSmall)
                                  : lp2d::kDefaultChunkSmall;
    p.check_finite = opt.check_finite ? 1 : 0;
}

}  // namespace

extern "C" {

int lp3d_solve_batch_ex(const float* ax, const float* ay, const float* az, const float* b, const int64_t* offsets,
                        int64_t n_lp, const float* obj_xyz, lp3d_box box, void* out_xyz, int32_t* out_status,
                        const lp2d_options* opt_in, void* workspace, size_t workspace_bytes, lp2d_stream_t stream) {
    using lp2d::report_error;
    lp2d_options opt;
    if (opt_in) opt = *opt_in;
    else lp2d_default_options(&opt);
    if (n_lp < 0) return report_error(LP2D_ERR_INVALID_ARGUMENT, "n_lp = %lld < 0", (long long)n_lp);
    int rc0 = check_options3(opt);
    if (rc0 != LP2D_OK) return rc0;
    const float bx[6] = {box.xmin, box.xmax, box.ymin, box.ymax, box.zmin, box.zmax};
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(bx[i])) return report_error(LP2D_ERR_INVALID_ARGUMENT, "box must be finite");
    if (!(box.xmin < box.xmax) || !(box.ymin < box.ymax) || !(box.zmin < box.zmax))
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "box needs min < max on every axis");
    if (n_lp == 0) return LP2D_OK;
    if (!ax || !ay || !az || !b || !offsets || !obj_xyz || !out_xyz || !out_status)
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "NULL data pointer");
    const size_t out_align = (opt.precision == LP2D_PREC_FP64) ? 8 : 4;
    if (!aligned3(ax, 4) || !aligned3(ay, 4) || !aligned3(az, 4) || !aligned3(b, 4) || !aligned3(obj_xyz, 4) ||
        !aligned3(offsets, 8) || !aligned3(out_xyz, out_align) || !aligned3(out_status, 4) ||
        (opt.out_nviol && !aligned3(opt.out_nviol, 4)) || (opt.out_def && !aligned3(opt.out_def, 4)))
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "misaligned pointer");
    const size_t need = sizeof(unsigned long long) * lp2d::kWsWords;
    if (!workspace) return report_error(LP2D_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", need);
    if (workspace_bytes < need || !aligned3(workspace, 8))
        return report_error(LP2D_ERR_WORKSPACE, "workspace needs %zu bytes, 8-byte aligned", need);

    lp2d::Params3 p{};
    p.ax = ax;
    p.ay = ay;
    p.az = az;
    p.b = b;
    p.offsets = offsets;
    p.n_lp = n_lp;
    p.obj = obj_xyz;
    for (int i = 0; i < 6; ++i) p.box[i] = bx[i];
    p.out_xyz = out_xyz;
    p.out_status = out_status;
    fill_common3(p, opt, workspace);
    return launch3(p, opt, n_lp, stream);
}

int lp2d_least_violation(const float* ax, const float* ay, const float* b, const int64_t* offsets, int64_t n_lp,
                         lp2d_box box, const int32_t* status_in, void* out_xy, float* out_t, int32_t* out_status,
                         const lp2d_options* opt_in, void* workspace, size_t workspace_bytes, lp2d_stream_t stream) {
    using lp2d::report_error;
    lp2d_options opt;
    if (opt_in) opt = *opt_in;
    else lp2d_default_options(&opt);
    if (n_lp < 0) return report_error(LP2D_ERR_INVALID_ARGUMENT, "n_lp = %lld < 0", (long long)n_lp);
    int rc0 = check_options3(opt);
    if (rc0 != LP2D_OK) return rc0;
    if (!std::isfinite(box.xmin) || !std::isfinite(box.xmax) || !std::isfinite(box.ymin) ||
        !std::isfinite(box.ymax) || !(box.xmin < box.xmax) || !(box.ymin < box.ymax))
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "box must be finite with xmin < xmax and ymin < ymax");
    if (n_lp == 0) return LP2D_OK;
    if (!ax || !ay || !b || !offsets || !status_in || !out_xy || !out_status)
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "NULL data pointer");
    const size_t out_align = (opt.precision == LP2D_PREC_FP64) ? 8 : 4;
    if (!aligned3(ax, 4) || !aligned3(ay, 4) || !aligned3(b, 4) || !aligned3(offsets, 8) ||
        !aligned3(status_in, 4) || !aligned3(out_xy, out_align) || (out_t && !aligned3(out_t, 4)) ||
        !aligned3(out_status, 4) || (opt.out_nviol && !aligned3(opt.out_nviol, 4)) ||
        (opt.out_def && !aligned3(opt.out_def, 4)))
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "misaligned pointer");
    const size_t need = sizeof(unsigned long long) * lp2d::kWsWords;
    if (!workspace) return report_error(LP2D_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", need);
    if (workspace_bytes < need || !aligned3(workspace, 8))
        return report_error(LP2D_ERR_WORKSPACE, "workspace needs %zu bytes, 8-byte aligned", need);
    const float bm = fmaxf(fmaxf(fabsf(box.xmin), fabsf(box.xmax)), fmaxf(fabsf(box.ymin), fabsf(box.ymax)));
    lp2d::Params3 p{};
    p.ax = ax;
    p.ay = ay;
    p.az = nullptr;
    p.b = b;
    p.offsets = offsets;
    p.n_lp = n_lp;
    p.obj = nullptr;
    p.box[0] = box.xmin;
    p.box[1] = box.xmax;
    p.box[2] = box.ymin;
    p.box[3] = box.ymax;
    p.box[4] = 0.0f;
    p.box[5] = LP2D_LEAST_VIOLATION_TMAX_FACTOR * bm;
    p.out_xyz = out_xy;
    p.out_status = out_status;
    p.status_in = status_in;
    p.out_t = out_t;
    fill_common3(p, opt, workspace);
    return launch3(p, opt, n_lp, stream);
}

}  // extern "C"
