// lp2d_warp.cuh -- Seidel's method (Sec. 2.1) on an LP staged in shared memory,
// driven by one warp, with the CTA's other warps joining long 1-D LPs.
//
// Stage layout (per LP, in visit order): slot s holds constraint (a_x, a_y) in a float2
// array and b in a float array, so that one 8-byte and one 4-byte shared-memory load
// fetch a constraint.  Slots 0..3 are the box sides (the +-M constraints of Sec. 2.1)
// x <= xmax, -x <= -xmin, y <= ymax, -y <= -ymin; slot 4 + p holds the constraint
// visited at position p.  Ties between equal sigma values go to the lowest slot, the
// earliest constraint, box first.
//
// Staging: every thread computes the visit-order keys E(q) of its constraints, marks
// them in a bitmap of the key domain (one shared-memory atomic OR each) and keeps
// them, two 16-bit keys per register; a prefix count of the bitmap words then gives
// each key its rank, the constraint's visit position, and cp.async copies a_x, a_y
// and b from HBM straight into that slot.
//
// Iteration: the warp tests the 32 positions of an aligned window against the current
// optimum; the first violated one (ballot) is the next step of serial Seidel, since
// every earlier position is satisfied.  After its 1-D LP the same window is tested
// again from the next position on, with the values still in registers, and the next
// window is loaded one step ahead.  The 1-D LP reduces sigma = num/den over slots
// 0 .. 4 + first - 1: den > 0 bounds t from the right (Eq. 4, min), den < 0 from the
// left (Eq. 3, max), den == 0 with num < 0 excludes the line.
#pragma once

#include "lp2d_device.cuh"
#include "lp2d_staged.cuh"

namespace lp2d {

// ------------------------------------------------------------------ primitives
// Bulk prefetch of the 16-byte-aligned interior of [p, p + n) into L2 (no bytes
// outside the range are touched).
__device__ __forceinline__ void prefetch_l2(const float* p, int64_t n) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uintptr_t e = reinterpret_cast<uintptr_t>(p + n);
    const uintptr_t a16 = (a + 15u) & ~static_cast<uintptr_t>(15);
    const uintptr_t e16 = e & ~static_cast<uintptr_t>(15);
    if (e16 > a16) {
        const unsigned bytes = static_cast<unsigned>(e16 - a16);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a16), "r"(bytes) : "memory");
    }
}

// Warp-wide reduction of a 1-D LP: (min right bound, its lowest slot), max left bound.
// FP32: the float min/max of redux.sync; FP64: butterfly shuffles on order-preserving
// 64-bit keys.  Every lane gets the result.
template <typename Real>
__device__ __forceinline__ void reduce_1dlp(Real& thi, int& phi, Real& tlo) {
    warp_reduce_1dlp<Real>(thi, phi, tlo);
}

// x * 0 is NaN exactly when x is NaN or infinite: folds the finiteness of a
// constraint into an accumulator that stays 0 for finite data.
__device__ __forceinline__ float fold_finite(float2 a, float b, float acc) {
    return fmaf(a.x, 0.0f, fmaf(a.y, 0.0f, fmaf(b, 0.0f, acc)));
}

// Barrier of a staging group: a warp, a pair of warps (named barrier `bar`), or the CTA.
// The pair barrier's id (3 or 4) is selected among immediates, so that the kernel
// declares only the barriers it uses.
__device__ __forceinline__ void pair_barrier(int bar) {
    if (bar == 3) asm volatile("bar.sync 3, 64;\n" ::: "memory");
    else asm volatile("bar.sync 4, 64;\n" ::: "memory");
}

template <int T>
__device__ __forceinline__ void group_sync(int bar) {
    if constexpr (T == 32) __syncwarp();
    else if constexpr (T == 64) pair_barrier(bar);
    else __syncthreads();
}

// Box sides into stage slots 0..3 (lanes 0..3 of the calling warp).
__device__ __forceinline__ void write_box2(const Params& P, float2* sA, float* sB, int lane) {
    if (lane < kBoxSlots) {
        const float gx = (lane == 0) ? 1.0f : (lane == 1) ? -1.0f : 0.0f;
        const float gy = (lane == 2) ? 1.0f : (lane == 3) ? -1.0f : 0.0f;
        sA[lane] = make_float2(gx, gy);
        sB[lane] = (lane == 0) ? P.xmax : (lane == 1) ? -P.xmin : (lane == 2) ? P.ymax : -P.ymin;
    }
}

// ------------------------------------------------------------------ staging
// T threads (one warp, a pair of warps, or the CTA's 128) stage the m constraints at
// gax/gay/gb into slots 4.. of sA/sB in visit order.  The key domain must fit NW
// bitmap words (NW = 32: m <= 1024; NW = 128: m <= 4096); threads 0..NW-1 own one
// word each.  bm, pre: NW words each (bm keeps the LP's key bitmap afterwards); wsum:
// NW/32 words.  Thread tid stages constraints tid, tid + T, ...; when there are at
// most KR of them per thread their keys are kept in registers between the two
// passes, otherwise they are computed again.  bar: the pair's named barrier (T = 64).
// Completion: cp_async_wait_all() then group_sync<T>(bar).
template <int T, int NW, int KR>
__device__ __forceinline__ void stage_lp2(const VisitOrder& vo, int m, const float* __restrict__ gax,
                                          const float* __restrict__ gay, const float* __restrict__ gb,
                                          float2* sA, float* sB, unsigned* bm, int* pre, int* wsum, int tid,
                                          int bar = 0) {
    static_assert((T == 32 && NW == 32) || (T == 64 && NW == 32) || (T == 128 && NW == 128), "staging group");
    const int lane = tid & 31;
    if (tid < NW) bm[tid] = 0u;
    group_sync<T>(bar);
    auto key_of = [&](int q) { return vo.enc(static_cast<uint32_t>(q)); };
    const bool keep = KR > 0 && m <= KR * T;
    uint32_t kk[KR > 0 ? (KR + 1) / 2 : 1];
#pragma unroll
    for (int i = 0; i < (KR + 1) / 2; ++i) kk[i] = 0u;
    if (keep) {
#pragma unroll
        for (int r = 0; r < KR; ++r) {
            if (T * r >= m) break;  // the same for every thread
            const int q = tid + T * r;
            if (q < m) {
                const uint32_t e = key_of(q);
                atomicOr(bm + (e >> 5), 1u << (e & 31u));
                kk[r >> 1] |= e << (16 * (r & 1));
            }
        }
    } else {
        for (int q = tid; q < m; q += T) {
            const uint32_t e = key_of(q);
            atomicOr(bm + (e >> 5), 1u << (e & 31u));
        }
    }
    group_sync<T>(bar);
    if (tid < NW) {  // whole warps
        const unsigned w = bm[tid];
        const int c = __popc(w);
        int incl = warp_inclusive_scan(c, lane);
        if constexpr (NW > 32) {
            if (lane == 31) wsum[tid >> 5] = incl;
            __syncthreads();
            int base = 0;
            for (int i = 0; i < (tid >> 5); ++i) base += wsum[i];
            incl += base;
        }
        pre[tid] = incl - c;
    }
    group_sync<T>(bar);
    // slot of key e: 4 + (number of smaller keys)
    auto slot_of = [&](uint32_t e) {
        const int wi = static_cast<int>(e >> 5);
        return kBoxSlots + pre[wi] + __popc(bm[wi] & ((1u << (e & 31u)) - 1u));
    };
    if (keep) {
#pragma unroll
        for (int r = 0; r < KR; ++r) {
            if (T * r >= m) break;
            const int q = tid + T * r;
            if (q < m) {
                const uint32_t e = (kk[r >> 1] >> (16 * (r & 1))) & 0xffffu;
                const int s = slot_of(e);
                cp_async4(&sA[s].x, gax + q);
                cp_async4(&sA[s].y, gay + q);
                cp_async4(sB + s, gb + q);
            }
        }
    } else {
        for (int q = tid; q < m; q += T) {
            const int s = slot_of(key_of(q));
            cp_async4(&sA[s].x, gax + q);
            cp_async4(&sA[s].y, gay + q);
            cp_async4(sB + s, gb + q);
        }
    }
}

// The LP's three constraint segments into L2 (one lane issues the bulk prefetches).
__device__ __forceinline__ void prefetch_lp(const Params& P, int64_t base, int64_t m, int lane) {
    if (lane == 0 && m > 0) {
        prefetch_l2(P.ax + base, m);
        prefetch_l2(P.ay + base, m);
        prefetch_l2(P.b + base, m);
    }
}

// ------------------------------------------------------------------ 1-D LP
// One lane's share of a 1-D LP: slots j0, j0 + STRIDE, ... below jend.  The line is
// p0 + t u with u oriented so that the objective's end is the right end: the right
// bound (min over den > 0, Eq. 4) is tracked with its slot, the left bound (max over
// den < 0, Eq. 3) by value only.  den is moved off -0 so that a constraint parallel
// to the line (den == 0) yields num / +0: -inf when it excludes the line (num < 0),
// which empties the interval, and +inf or NaN (no effect) when it does not.
// kFlag: also report (in *np) whether a work unit had near-parallel normals,
// den^2 < lim |g|^2; kMixed: recompute such work units in FP64 (the products of the
// FP32 inputs are exact there).
template <typename Real, int STRIDE, bool kFlag = false, bool kMixed = false>
__device__ __forceinline__ void wu_range2(const float2* __restrict__ sA, const float* __restrict__ sB, int j0,
                                          int jend, Real p0x, Real p0y, Real ux, Real uy, Real& thi, int& phi,
                                          Real& tlo, const MixedLine& ml = MixedLine{0.0, 0.0, 0.0f},
                                          bool* np = nullptr) {
    const Real ninf = -real_inf<Real>();
    bool near = false;
#pragma unroll 4
    for (int j = j0; j < jend; j += STRIDE) {
        const float2 g = sA[j];
        const Real gx = g.x, gy = g.y, gb = sB[j];
        Real den, num;
        if constexpr (sizeof(Real) == 4 && !kFlag && !kMixed) {
            // fused forms: the inner fma's +0 addend keeps den off -0 (an exact zero
            // sum rounds to +0), as the + 0 below does
            den = fmaf(gx, ux, fmaf(gy, uy, 0.0f));
            num = fmaf(-gx, p0x, fmaf(-gy, p0y, gb));
        } else {
            den = (gx * ux + gy * uy) + Real(0);
            num = gb - (gx * p0x + gy * p0y);
        }
        Real t = real_div<Real>(num, den);
        if constexpr (kFlag || kMixed) {
            const bool is_near = den * den < ml.lim * (gx * gx + gy * gy);
            if constexpr (kFlag) near = near || is_near;
            if constexpr (kMixed) {
                if (is_near) {
                    // + 0.0 turns -0 into +0, as for den above: num / +0 is the parallel case
                    const double d64 = (static_cast<double>(gx) * static_cast<double>(ux) +
                                        static_cast<double>(gy) * static_cast<double>(uy)) + 0.0;
                    const double n64 = static_cast<double>(gb) -
                                       (static_cast<double>(gx) * ml.p0x + static_cast<double>(gy) * ml.p0y);
                    t = static_cast<Real>(n64 / d64);
                    den = (d64 < 0.0) ? Real(-1) : Real(1);
                }
            }
        }
        const bool right = den >= Real(0);
        const bool take = right && (t < thi);
        thi = take ? t : thi;
        phi = take ? j : phi;
        tlo = real_max<Real>(tlo, right ? ninf : t);
    }
    if constexpr (kFlag) *np = near;
}

// Shared-memory protocol between the driving warp and its three helpers.
template <typename Real>
struct TeamJob2 {
    int cmd;    // kJobRun or kJobDone
    int fslot;  // slots 0 .. fslot-1 take part
    Real p0x, p0y, ux, uy;
    double p0x64, p0y64;  // the FP64 foot of the line (mixed precision)
    float lim;            // near-parallel threshold of the mixed-precision mode
    Real thi[4], tlo[4];
    int phi[4];
};

// Helpers (the CTA's warps other than the driver): wait for jobs until kJobDone.
template <typename Real, bool kMixed>
__device__ void team_helper2(const float2* __restrict__ sA, const float* __restrict__ sB, TeamJob2<Real>* job,
                             int tid) {
    const int warp = tid >> 5, lane = tid & 31;
    for (;;) {
        named_barrier(kTeamBarJob, kTeamThreads);
        if (job->cmd != kJobRun) break;
        Real thi = real_inf<Real>(), tlo = -real_inf<Real>();
        int phi = kNoPos;
        const MixedLine ml{job->p0x64, job->p0y64, job->lim};
        wu_range2<Real, kTeamThreads, false, kMixed>(sA, sB, tid, job->fslot, job->p0x, job->p0y, job->ux, job->uy,
                                                     thi, phi, tlo, ml);
        reduce_1dlp(thi, phi, tlo);
        if (lane == 0) {
            job->thi[warp] = thi;
            job->tlo[warp] = tlo;
            job->phi[warp] = phi;
        }
        named_barrier(kTeamBarPart, kTeamThreads);
    }
}

// ------------------------------------------------------------------ the driver
// Seidel's iterations over one staged LP by one warp (lane = 0..31).  With a team
// (kTeam), 1-D LPs over at least P.team_min slots are shared with the helper warps,
// and the driver posts kJobDone when it has finished.  Writes the LP's outputs.
template <typename Real, bool kMixed, bool kTeam>
__device__ void drive_lp2(const Params& P, int64_t lp, int m, float cxf, float cyf, const VisitOrder& vo,
                          const float2* __restrict__ sA, const float* __restrict__ sB, const unsigned* bm, int lane,
                          TeamJob2<Real>* job) {
    const Real cx = static_cast<Real>(cxf), cy = static_cast<Real>(cyf);
    const Real eps = (sizeof(Real) == 4) ? Real(P.eps32) : Real(P.eps64);
    Real vx = (cx >= Real(0)) ? Real(P.xmax) : Real(P.xmin);
    Real vy = (cy >= Real(0)) ? Real(P.ymax) : Real(P.ymin);
    Real avx = real_abs(vx), avy = real_abs(vy);
    int d0 = (cx >= Real(0)) ? 0 : 1;  // slots of the defining pair
    int d1 = (cy >= Real(0)) ? 2 : 3;
    int status = -1;
    int nviol = 0;
    float fin = 0.0f;
    // window [k, k + 32): lane l holds position k + l in (ca, cb); positions below kmin
    // are known to be satisfied.  (na, nb) is the next window, loaded a step ahead.
    int k = 0, kmin = 0;
    float2 ca = make_float2(0.0f, 0.0f), na = make_float2(0.0f, 0.0f);
    float cb = 0.0f, nb = 0.0f;
    if (lane < m) {
        ca = sA[kBoxSlots + lane];
        cb = sB[kBoxSlots + lane];
    }
    if (32 + lane < m) {
        na = sA[kBoxSlots + 32 + lane];
        nb = sB[kBoxSlots + 32 + lane];
    }
    fin = fold_finite(ca, cb, fold_finite(na, nb, fin));
    while (k < m) {
        const int p = k + lane;
        bool viol = false;
        if (p < m && p >= kmin) {
            const Real gx = ca.x, gy = ca.y, gb = cb;
            const Real s = gx * vx + gy * vy - gb;
            const Real tol = eps * (real_abs(gx) * avx + real_abs(gy) * avy + real_abs(gb));
            viol = s > tol;
        }
        const unsigned bal = __ballot_sync(kFull, viol);
        if (bal == 0u) {
            k += 32;
            ca = na;
            cb = nb;
            if (k + 32 + lane < m) {
                na = sA[kBoxSlots + k + 32 + lane];
                nb = sB[kBoxSlots + k + 32 + lane];
                fin = fold_finite(na, nb, fin);
            }
            continue;
        }
        const int first = k + __ffs(bal) - 1;
        const int fslot = kBoxSlots + first;
        kmin = first + 1;
        // ---- 1-D LP on the violated line l: lx*x + ly*y = lb
        const float2 la = sA[fslot];
        const Real lx = la.x, ly = la.y, lb = sB[fslot];
        const Real nrm2 = lx * lx + ly * ly;
        if (!(nrm2 != Real(0))) {  // 0.x <= lb < 0 (NaN data also stops here)
            status = kInfeasible;
            break;
        }
        const Real sc0 = real_div<Real>(lb, nrm2);
        const Real p0x = lx * sc0, p0y = ly * sc0;  // foot of l
        // Direction of l, oriented so that the objective's end is the right end; when
        // c.u == 0 the left end of u = (-ly, lx) is taken.
        const Real cu = cx * (-ly) + cy * lx;
        const Real fs = (cu > Real(0)) ? Real(1) : Real(-1);
        const Real ux = -ly * fs, uy = lx * fs;
        MixedLine ml{0.0, 0.0, 0.0f};
        // the foot of l in FP64, computed only when a near-parallel pair or a grazing
        // interval needs it (FP64 division is slow on this GPU)
        auto foot64 = [&]() {
            const double lx64 = lx, ly64 = ly, sc64 = static_cast<double>(lb) / (lx64 * lx64 + ly64 * ly64);
            ml.p0x = lx64 * sc64;
            ml.p0y = ly64 * sc64;
        };
        if constexpr (kMixed) ml.lim = P.tau * P.tau * static_cast<float>(nrm2);
        Real thi = real_inf<Real>(), tlo = -real_inf<Real>();
        int phi = kNoPos;
        if (kTeam && fslot >= P.team_min) {
            if constexpr (kMixed) foot64();
            if (lane == 0) {
                job->cmd = kJobRun;
                job->fslot = fslot;
                job->p0x = p0x;
                job->p0y = p0y;
                job->ux = ux;
                job->uy = uy;
                job->p0x64 = ml.p0x;
                job->p0y64 = ml.p0y;
                job->lim = ml.lim;
            }
            named_barrier(kTeamBarJob, kTeamThreads);
            // the driver takes the slots of its own thread index, like every helper
            wu_range2<Real, kTeamThreads, false, kMixed>(sA, sB, static_cast<int>(threadIdx.x), fslot, p0x, p0y, ux,
                                                         uy, thi, phi, tlo, ml);
            reduce_1dlp(thi, phi, tlo);
            named_barrier(kTeamBarPart, kTeamThreads);
            const int self = static_cast<int>(threadIdx.x >> 5);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (w == self) continue;
                const Real th = job->thi[w];
                const int ph = job->phi[w];
                if (th < thi || (th == thi && ph < phi)) {
                    thi = th;
                    phi = ph;
                }
                tlo = real_max<Real>(tlo, job->tlo[w]);
            }
        } else if (!kMixed && fslot <= 32) {
            // a short 1-D LP: one slot per lane, no loop
            if (lane < fslot) {
                const float2 g = sA[lane];
                const Real gx = g.x, gy = g.y, gb = sB[lane];
                const Real den = (gx * ux + gy * uy) + Real(0);
                const Real num = gb - (gx * p0x + gy * p0y);
                const Real t = real_div<Real>(num, den);
                const bool right = den >= Real(0);
                if (right && t < thi) {
                    thi = t;
                    phi = lane;
                }
                tlo = right ? tlo : t;
            }
            reduce_1dlp(thi, phi, tlo);
        } else if (!kMixed && fslot <= 64) {
            // a short 1-D LP: at most two slots per lane, no loop
            const Real ninf = -real_inf<Real>();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                if (j < fslot) {
                    const float2 g = sA[j];
                    const Real gx = g.x, gy = g.y, gb = sB[j];
                    const Real den = (gx * ux + gy * uy) + Real(0);
                    const Real num = gb - (gx * p0x + gy * p0y);
                    const Real t = real_div<Real>(num, den);
                    const bool right = den >= Real(0);
                    const bool take = right && (t < thi);
                    thi = take ? t : thi;
                    phi = take ? j : phi;
                    tlo = real_max<Real>(tlo, right ? ninf : t);
                }
            }
            reduce_1dlp(thi, phi, tlo);
        } else {
            bool np = false;
            wu_range2<Real, 32, kMixed>(sA, sB, lane, fslot, p0x, p0y, ux, uy, thi, phi, tlo, ml, &np);
            if (kMixed && __any_sync(kFull, np)) {
                // a near-parallel pair: redo this 1-D LP with FP64 intersections for them
                foot64();
                thi = real_inf<Real>();
                tlo = -real_inf<Real>();
                phi = kNoPos;
                wu_range2<Real, 32, false, kMixed>(sA, sB, lane, fslot, p0x, p0y, ux, uy, thi, phi, tlo, ml);
            }
            reduce_1dlp(thi, phi, tlo);
        }
        ++nviol;
        bool empty = !(tlo <= thi);  // an excluding parallel constraint makes thi = -inf
        Real nvx = p0x + thi * ux, nvy = p0y + thi * uy;
        if constexpr (kMixed) {
            // a grazing interval (ends within FP32 rounding of each other): decide the
            // 1-D LP again in FP64 before trusting emptiness or the endpoint
            if (!empty && (thi - tlo) <= Real(1e-5) * (real_abs(thi) + real_abs(tlo) + Real(1))) {
                foot64();
                double th64 = real_inf<double>(), tl64 = -real_inf<double>();
                int ph64 = kNoPos;
                wu_range2<double, 32>(sA, sB, lane, fslot, ml.p0x, ml.p0y, static_cast<double>(ux),
                                      static_cast<double>(uy), th64, ph64, tl64);
                reduce_1dlp(th64, ph64, tl64);
                empty = !(tl64 <= th64);
                phi = ph64;
                nvx = static_cast<Real>(ml.p0x + th64 * static_cast<double>(ux));
                nvy = static_cast<Real>(ml.p0y + th64 * static_cast<double>(uy));
            }
        }
        if (empty) {
            status = kInfeasible;
            break;
        }
        vx = nvx;
        vy = nvy;
        avx = real_abs(vx);
        avy = real_abs(vy);
        d0 = fslot;
        d1 = phi;
    }
    // positions never loaded (the LP stopped early) still take part in the finiteness check
    if (P.check_finite) {
        for (int p = k + 64 + lane; p < m; p += 32)
            fin = fold_finite(sA[kBoxSlots + p], sB[kBoxSlots + p], fin);
    }
    const bool bad_data = P.check_finite && __any_sync(kFull, fin != fin);
    const bool bad_obj = !(fabsf(cxf) <= 3.402823466e38f) || !(fabsf(cyf) <= 3.402823466e38f);
    int id0 = 0, id1 = 0;
    if (P.out_def) {  // warp-uniform; the key bitmap is still intact
        id0 = slot_id(d0, vo, bm, lane);
        id1 = slot_id(d1, vo, bm, lane);
    }
    if constexpr (kTeam) {
        if (lane == 0) job->cmd = kJobDone;
        named_barrier(kTeamBarJob, kTeamThreads);
    }
    if (lane == 0) {
        if (bad_data || bad_obj) status = kBadInput;
        else if (status < 0) status = (d0 < kBoxSlots || d1 < kBoxSlots) ? kBoxBounded : kOptimal;
        Real* out = reinterpret_cast<Real*>(P.out_xy);
        if (status == kInfeasible || status == kBadInput) {
            const Real nan = real_inf<Real>() - real_inf<Real>();
            out[2 * lp] = nan;
            out[2 * lp + 1] = nan;
        } else {
            out[2 * lp] = vx;
            out[2 * lp + 1] = vy;
        }
        P.out_status[lp] = status;
        if (P.out_nviol) P.out_nviol[lp] = nviol;
        if (P.out_def) {
            P.out_def[2 * lp] = id0;
            P.out_def[2 * lp + 1] = id1;
        }
    }
}

// ------------------------------------------------------------------ FP32 driver
// The FP32 iterations of drive_lp2 with fewer instructions per step: positions past
// the LP hold an inert constraint (0, 0, FLT_MAX) that no optimum violates, so the
// window test needs no range check; the lanes of a window already known to be
// satisfied are masked out of its ballot; the violated line comes from the lane that
// holds it; the tolerance terms eps |v_x| and eps |v_y| change only with the vertex.
constexpr float kInertB = 3.402823466e38f;

__device__ __forceinline__ void load_window(const float2* __restrict__ sA, const float* __restrict__ sB, int q, int m,
                                            float2& a, float& b) {
    if (q < m) {
        a = sA[kBoxSlots + q];
        b = sB[kBoxSlots + q];
    } else {
        a = make_float2(0.0f, 0.0f);
        b = kInertB;
    }
}

// H: the warp tests 32 H positions per step (H rows of 32, lane l holding positions
// k + 32 h + l), which halves the serial steps of long violation-free stretches at
// H = 2.
template <bool kTeam, int H, bool kAhead = true>
__device__ void drive_f32(const Params& P, int64_t lp, int m, float cx, float cy, const VisitOrder& vo,
                          const float2* __restrict__ sA, const float* __restrict__ sB, const unsigned* bm, int lane,
                          TeamJob2<float>* job) {
    static_assert(H >= 1 && H <= 4, "one to four rows per window");
    constexpr int kW = 32 * H;  // positions per window
    const float eps = P.eps32;
    float vx = (cx >= 0.0f) ? P.xmax : P.xmin;
    float vy = (cy >= 0.0f) ? P.ymax : P.ymin;
    float ex = eps * fabsf(vx), ey = eps * fabsf(vy);
    int d0 = (cx >= 0.0f) ? 0 : 1;  // slots of the defining pair
    int d1 = (cy >= 0.0f) ? 2 : 3;
    int status = -1;
    int nviol = 0;
    // window [k, k + kW): row h of lane l holds position k + 32 h + l in (ca[h], cb[h]);
    // live[h] marks the lanes of row h not yet known to be satisfied; (na, nb) is the
    // next window.
    int k = 0;
    unsigned live[H];
    float2 ca[H], na[H];
    float cb[H], nb[H];
    float fin = 0.0f;
#pragma unroll
    for (int h = 0; h < H; ++h) {
        live[h] = kFull;
        load_window(sA, sB, 32 * h + lane, m, ca[h], cb[h]);
        fin = fold_finite(ca[h], cb[h], fin);
        if constexpr (kAhead) {
            load_window(sA, sB, kW + 32 * h + lane, m, na[h], nb[h]);
            fin = fold_finite(na[h], nb[h], fin);
        }
    }
    for (;;) {
        unsigned bal[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const float s = fmaf(ca[h].x, vx, fmaf(ca[h].y, vy, -cb[h]));
            const float tol = fmaf(fabsf(ca[h].x), ex, fmaf(fabsf(ca[h].y), ey, eps * fabsf(cb[h])));
            bal[h] = __ballot_sync(kFull, s > tol) & live[h];
        }
        // the first row with a violation (hv) and its ballot (bv)
        int hv = 0;
        unsigned bv = bal[0];
#pragma unroll
        for (int h = H - 1; h >= 1; --h) {
            if (bal[h] != 0u && bal[0] == 0u) {
                bool earlier = false;
#pragma unroll
                for (int g = 1; g < h; ++g) earlier = earlier || bal[g] != 0u;
                if (!earlier) {
                    hv = h;
                    bv = bal[h];
                }
            }
        }
        if (bv == 0u) {
            k += kW;
            if (k >= m) break;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                live[h] = kFull;
                if constexpr (kAhead) {
                    ca[h] = na[h];
                    cb[h] = nb[h];
                    load_window(sA, sB, k + kW + 32 * h + lane, m, na[h], nb[h]);
                    fin = fold_finite(na[h], nb[h], fin);
                } else {
                    load_window(sA, sB, k + 32 * h + lane, m, ca[h], cb[h]);
                    fin = fold_finite(ca[h], cb[h], fin);
                }
            }
            continue;
        }
        const int src = __ffs(bv) - 1;
#pragma unroll
        for (int h = 0; h < H; ++h) {
            if (h < hv) live[h] = 0u;
            else if (h == hv) live[h] = ~((2u << src) - 1u);  // lanes above src (none when src = 31)
        }
        const int fslot = kBoxSlots + k + 32 * hv + src;
        // ---- 1-D LP on the violated line l: lx*x + ly*y = lb
        float2 rowa = ca[0];
        float rowb = cb[0];
#pragma unroll
        for (int h = 1; h < H; ++h) {
            if (hv == h) {
                rowa = ca[h];
                rowb = cb[h];
            }
        }
        const float lx = __shfl_sync(kFull, rowa.x, src);
        const float ly = __shfl_sync(kFull, rowa.y, src);
        const float lb = __shfl_sync(kFull, rowb, src);
        const float nrm2 = fmaf(lx, lx, ly * ly);  // the lane-group driver's forms
        if (!(nrm2 != 0.0f)) {  // 0.x <= lb < 0 (NaN data also stops here)
            status = kInfeasible;
            break;
        }
        const float sc0 = __fdividef(lb, nrm2);
        const float p0x = lx * sc0, p0y = ly * sc0;  // foot of l
        // direction of l, oriented so that the objective's end is the right end; when
        // c.u == 0 the left end of u = (-ly, lx) is taken
        const float cu = fmaf(cx, -ly, cy * lx);
        const float ux = (cu > 0.0f) ? -ly : ly;
        const float uy = (cu > 0.0f) ? lx : -lx;
        float thi = real_inf<float>(), tlo = -real_inf<float>();
        int phi = kNoPos;
        if (kTeam && fslot >= P.team_min) {
            if (lane == 0) {
                job->cmd = kJobRun;
                job->fslot = fslot;
                job->p0x = p0x;
                job->p0y = p0y;
                job->ux = ux;
                job->uy = uy;
            }
            named_barrier(kTeamBarJob, kTeamThreads);
            wu_range2<float, kTeamThreads>(sA, sB, static_cast<int>(threadIdx.x), fslot, p0x, p0y, ux, uy, thi, phi,
                                           tlo);
            reduce_1dlp(thi, phi, tlo);
            named_barrier(kTeamBarPart, kTeamThreads);
            const int self = static_cast<int>(threadIdx.x >> 5);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (w == self) continue;
                const float th = job->thi[w];
                const int ph = job->phi[w];
                if (th < thi || (th == thi && ph < phi)) {
                    thi = th;
                    phi = ph;
                }
                tlo = fmaxf(tlo, job->tlo[w]);
            }
        } else {
            if (fslot <= 32) {
                // a short 1-D LP: one slot per lane, no loop; lanes at or past fslot
                // load a later slot of the stage and ignore it
                const float2 g = sA[lane];
                const float gb = sB[lane];
                const float den = fmaf(g.x, ux, fmaf(g.y, uy, 0.0f));
                const float t = __fdividef(fmaf(-g.x, p0x, fmaf(-g.y, p0y, gb)), den);
                const bool in = lane < fslot;
                const bool right = den >= 0.0f;
                if (in && right && t < thi) {  // t is NaN for 0 / 0: no bound
                    thi = t;
                    phi = lane;
                }
                tlo = (in && !right) ? t : tlo;
            } else {
                wu_range2<float, 32>(sA, sB, lane, fslot, p0x, p0y, ux, uy, thi, phi, tlo);
            }
            reduce_1dlp(thi, phi, tlo);
        }
        ++nviol;
        if (!(tlo <= thi)) {  // empty interval; an excluding parallel constraint makes thi = -inf
            status = kInfeasible;
            break;
        }
        vx = fmaf(thi, ux, p0x);
        vy = fmaf(thi, uy, p0y);
        ex = eps * fabsf(vx);
        ey = eps * fabsf(vy);
        d0 = fslot;
        d1 = phi;
    }
    // positions never loaded (the LP stopped early) still take part in the finiteness check
    if (P.check_finite) {
        for (int p = k + (kAhead ? 2 : 1) * kW + lane; p < m; p += 32)
            fin = fold_finite(sA[kBoxSlots + p], sB[kBoxSlots + p], fin);
    }
    const bool bad_data = P.check_finite && __any_sync(kFull, fin != fin);
    const bool bad_obj = !(fabsf(cx) <= 3.402823466e38f) || !(fabsf(cy) <= 3.402823466e38f);
    int id0 = 0, id1 = 0;
    if (P.out_def) {  // warp-uniform; the key bitmap is still intact
        id0 = slot_id(d0, vo, bm, lane);
        id1 = slot_id(d1, vo, bm, lane);
    }
    if constexpr (kTeam) {
        if (lane == 0) job->cmd = kJobDone;
        named_barrier(kTeamBarJob, kTeamThreads);
    }
    if (lane == 0) {
        if (bad_data || bad_obj) status = kBadInput;
        else if (status < 0) status = (d0 < kBoxSlots || d1 < kBoxSlots) ? kBoxBounded : kOptimal;
        float* out = reinterpret_cast<float*>(P.out_xy);  // 4-byte aligned only
        const bool none = status == kInfeasible || status == kBadInput;
        const float nan = real_inf<float>() - real_inf<float>();
        out[2 * lp] = none ? nan : vx;
        out[2 * lp + 1] = none ? nan : vy;
        P.out_status[lp] = status;
        if (P.out_nviol) P.out_nviol[lp] = nviol;
        if (P.out_def) {
            P.out_def[2 * lp] = id0;
            P.out_def[2 * lp + 1] = id1;
        }
    }
}

}  // namespace lp2d
