// lp2d_lane.cuh -- one lane per LP for the smallest LPs (FP32).
//
// The paper maps one thread to one LP (Sec. 3) and reads each constraint from global
// memory whenever a 1-D LP needs it.  Here that mapping is kept for LPs of at most
// kLaneCap constraints, 32 of them per warp, but each lane first copies its LP into
// the warp's part of the stage in visit order, interleaved by lane (the constraint at
// position p of lane l in slot 32 p + l, so that the lanes' reads fall in distinct
// banks), and then runs Seidel's iterations over it on its own: no ballot, shuffle or
// reduction, where a whole warp on such an LP spends most of its instructions on those.  The visit
// order, the tolerance, the 1-D LP arithmetic and the tie rules (box first, then the
// earliest position) are the one-warp driver's (drive_f32), so every result is
// bit-identical to the one a warp computes.
#pragma once

#include "lp2d_warp.cuh"

namespace lp2d {

constexpr int kLaneCap = 16;  // largest LP: a key domain of at most 16 keys, a visit order of 16 nibbles

// Position of the n-th (from 0) set bit of x, which has more than n set bits: the
// largest p with popc(x below p) <= n.
__device__ __forceinline__ int nth_set_bit(unsigned x, int n) {
    int p = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1)
        if (__popc(x & ((1u << (p + s)) - 1u)) <= n) p += s;
    return p;
}

// The calling lane copies its LP's m <= kLaneCap constraints into slots 32 p + lane of
// sA / sB in visit order (p: the visit position), by a scan of the key domain (4 or 16
// keys) in increasing order; returns the visit order, nibble p holding the constraint
// at position p.  Completion: cp_async_wait_all() then __syncwarp().
__device__ __forceinline__ uint64_t stage_lane(const VisitOrder& vo, int m, const float* __restrict__ gax,
                                               const float* __restrict__ gay, const float* __restrict__ gb,
                                               float2* sA, float* sB, int lane) {
    const uint32_t dom = static_cast<uint32_t>(vo.domain());
    uint64_t ord = 0;
    int n = 0;
    for (uint32_t e = 0; e < dom; ++e) {
        const uint32_t q = vo.dec(e);
        if (q < static_cast<uint32_t>(m)) {
            const int s = 32 * n + lane;
            cp_async4(&sA[s].x, gax + q);
            cp_async4(&sA[s].y, gay + q);
            cp_async4(sB + s, gb + q);
            ord |= static_cast<uint64_t>(q) << (4 * n);
            ++n;
        }
    }
    return ord;
}

// One step of the lane's 1-D LP: the work unit of stage slot `slot` with normal
// (gx, gy) and offset gb, in the forms of drive_f32 (the right bound keeps its slot
// on strict improvement, so the earliest slot wins a tie).
__device__ __forceinline__ void lane_unit(float gx, float gy, float gb, int slot, float p0x, float p0y, float ux,
                                          float uy, float& thi, int& phi, float& tlo) {
    const float den = fmaf(gx, ux, fmaf(gy, uy, 0.0f));
    const float t = __fdividef(fmaf(-gx, p0x, fmaf(-gy, p0y, gb)), den);
    const bool right = den >= 0.0f;
    if (right && t < thi) {
        thi = t;
        phi = slot;
    }
    tlo = fmaxf(tlo, right ? -real_inf<float>() : t);
}

// Seidel's iterations of LP lp (m <= kLaneCap constraints, staged by stage_lane with
// visit order ord) by the calling lane alone.  valid = false: the lane has no LP and
// writes nothing.
__device__ void solve_lane_f32(const Params& P, int64_t lp, bool valid, int m, float cx, float cy, uint64_t ord,
                               const float2* __restrict__ sA, const float* __restrict__ sB, int lane) {
    if (!valid) return;
    auto at = [&](int p) { return 32 * p + lane; };
    const float eps = P.eps32;
    float vx = (cx >= 0.0f) ? P.xmax : P.xmin;
    float vy = (cy >= 0.0f) ? P.ymax : P.ymin;
    float ex = eps * fabsf(vx), ey = eps * fabsf(vy);
    int d0 = (cx >= 0.0f) ? 0 : 1;
    int d1 = (cy >= 0.0f) ? 2 : 3;
    int status = -1;
    int nviol = 0;
    float fin = 0.0f;
    int p = 0;
    for (; p < m; ++p) {
        const float2 a = sA[at(p)];
        const float b = sB[at(p)];
        fin = fold_finite(a, b, fin);
        const float s = fmaf(a.x, vx, fmaf(a.y, vy, -b));
        const float tol = fmaf(fabsf(a.x), ex, fmaf(fabsf(a.y), ey, eps * fabsf(b)));
        if (!(s > tol)) continue;
        // the 1-D LP on the violated line over the box (slots 0..3) and positions 0..p-1
        const float nrm2 = fmaf(a.x, a.x, a.y * a.y);
        if (!(nrm2 != 0.0f)) {  // 0.x <= b < 0
            status = kInfeasible;
            break;
        }
        const float sc0 = __fdividef(b, nrm2);
        const float p0x = a.x * sc0, p0y = a.y * sc0;
        const float cu = fmaf(cx, -a.y, cy * a.x);
        const float ux = (cu > 0.0f) ? -a.y : a.y;
        const float uy = (cu > 0.0f) ? a.x : -a.x;
        float thi = real_inf<float>(), tlo = -real_inf<float>();
        int phi = kNoPos;
        lane_unit(1.0f, 0.0f, P.xmax, 0, p0x, p0y, ux, uy, thi, phi, tlo);
        lane_unit(-1.0f, 0.0f, -P.xmin, 1, p0x, p0y, ux, uy, thi, phi, tlo);
        lane_unit(0.0f, 1.0f, P.ymax, 2, p0x, p0y, ux, uy, thi, phi, tlo);
        lane_unit(0.0f, -1.0f, -P.ymin, 3, p0x, p0y, ux, uy, thi, phi, tlo);
        for (int j = 0; j < p; ++j) {
            const float2 g = sA[at(j)];
            lane_unit(g.x, g.y, sB[at(j)], kBoxSlots + j, p0x, p0y, ux, uy, thi, phi, tlo);
        }
        ++nviol;
        if (!(tlo <= thi)) {  // empty interval
            status = kInfeasible;
            break;
        }
        vx = fmaf(thi, ux, p0x);
        vy = fmaf(thi, uy, p0y);
        ex = eps * fabsf(vx);
        ey = eps * fabsf(vy);
        d0 = kBoxSlots + p;
        d1 = phi;
    }
    // positions never visited (the LP stopped early) take part in the finiteness check
    if (P.check_finite)
        for (int r = p + 1; r < m; ++r) fin = fold_finite(sA[at(r)], sB[at(r)], fin);
    const bool bad = (P.check_finite && fin != fin) || !(fabsf(cx) <= 3.402823466e38f) ||
                     !(fabsf(cy) <= 3.402823466e38f);
    if (bad) status = kBadInput;
    else if (status < 0) status = (d0 < kBoxSlots || d1 < kBoxSlots) ? kBoxBounded : kOptimal;
    float* out = reinterpret_cast<float*>(P.out_xy);
    const bool none = status == kInfeasible || status == kBadInput;
    const float nan = real_inf<float>() - real_inf<float>();
    out[2 * lp] = none ? nan : vx;
    out[2 * lp + 1] = none ? nan : vy;
    P.out_status[lp] = status;
    if (P.out_nviol) P.out_nviol[lp] = nviol;
    if (P.out_def) {
        auto id = [&](int slot) {
            return slot < kBoxSlots ? -1 - slot : static_cast<int>((ord >> (4 * (slot - kBoxSlots))) & 15u);
        };
        P.out_def[2 * lp] = id(d0);
        P.out_def[2 * lp + 1] = id(d1);
    }
}

}  // namespace lp2d
