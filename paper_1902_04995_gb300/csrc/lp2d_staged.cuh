// lp2d_staged.cuh -- Seidel's method on an LP staged in shared memory, solved by one
// warp, or by one warp with three helper warps for the long 1-D LPs.
//
// Stage layout (per LP, in visit order): slots 0..3 hold the four box sides (the +-M
// constraints of Sec. 2.1) in the order x <= xmax, -x <= -xmin, y <= ymax, -y <= -ymin;
// slot 4 + p holds the constraint visited at position p.  A slot index is therefore a
// visit position shifted by 4, and ties between equal sigma values go to the lowest
// slot -- the earliest constraint, box first.
//
// Staging: the keys E(q) of all constraints are set in a bitmap of the key domain
// (one shared-memory atomic OR each); a prefix count of the bitmap words gives every
// key its rank, which is the constraint's visit position.  Each constraint is then
// copied from HBM straight to its stage slot by asynchronous 4-byte copies
// (cp.async): global reads stay coalesced, no register holds the data, and no lane
// loops longer than another.
//
// Iteration (Sec. 2.1): the warp tests 32 consecutive positions against the current
// optimum at once; the first violated position (ballot) is the next step of serial
// Seidel, since every earlier position is satisfied.  Its 1-D LP reduces
// sigma = num/den over slots 0 .. 4+first-1: den > 0 bounds t from the right
// (Eq. 4, min), den < 0 from the left (Eq. 3, max), den == 0 with num < 0 excludes
// the line.  Lanes reduce strided slots, then redux.sync reduces (key, slot) pairs.
#pragma once

#include "lp2d_device.cuh"

namespace lp2d {

constexpr int kBoxSlots = 4;
constexpr int kWuUnroll = 2;    // unrolling of the 1-D LP loop

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gsrc) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void named_barrier(int id, int count) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

// SplitMix64 round keys: lanes 0..3 compute one output each, the warp shares them.
__device__ __forceinline__ void warp_visit_order(VisitOrder& vo, uint64_t seed, uint32_t m, int lane) {
    vo.init_shape(m);
    const uint32_t mine = static_cast<uint32_t>(splitmix64_output(seed, static_cast<uint32_t>(lane & 3)));
    vo.k0 = __shfl_sync(kFull, mine, 0);
    vo.k1 = __shfl_sync(kFull, mine, 1);
    vo.k2 = __shfl_sync(kFull, mine, 2);
    vo.k3 = __shfl_sync(kFull, mine, 3);
}

// Box sides into stage slots 0..3 (lanes 0..3 of the calling warp).
__device__ __forceinline__ void write_box(const Params& P, float* sX, float* sY, float* sB, int lane) {
    if (lane < kBoxSlots) {
        sX[lane] = (lane == 0) ? 1.0f : (lane == 1) ? -1.0f : 0.0f;
        sY[lane] = (lane == 2) ? 1.0f : (lane == 3) ? -1.0f : 0.0f;
        sB[lane] = (lane == 0) ? P.xmax : (lane == 1) ? -P.xmin : (lane == 2) ? P.ymax : -P.ymin;
    }
}

__device__ __forceinline__ int warp_inclusive_scan(int v, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int n = __shfl_up_sync(kFull, v, off);
        if (lane >= off) v += n;
    }
    return v;
}

__device__ __forceinline__ void stage_copy(int slot, int q, const float* __restrict__ gax,
                                           const float* __restrict__ gay, const float* __restrict__ gb,
                                           float* sX, float* sY, float* sB) {
    cp_async4(sX + slot, gax + q);
    cp_async4(sY + slot, gay + q);
    cp_async4(sB + slot, gb + q);
}

// Warp staging of an LP with m <= 1024 constraints (key domain <= 1024 bits, one
// bitmap word per lane).  bm: 32 words of shared memory owned by the warp; it keeps
// the LP's key bitmap afterwards.  Completion: cp_async_wait_all() then __syncwarp().
__device__ __forceinline__ void stage_lp_warp(const VisitOrder& vo, int m, const float* __restrict__ gax,
                                              const float* __restrict__ gay, const float* __restrict__ gb,
                                              float* sX, float* sY, float* sB, unsigned* bm, int lane) {
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
        if (valid) stage_copy(kBoxSlots + pe + __popc(we & ((1u << (e & 31u)) - 1u)), q, gax, gay, gb, sX, sY, sB);
    }
}

// CTA staging (4 warps) of an LP with m <= 4096 constraints (key domain <= 4096 bits,
// one bitmap word per thread).  bm, pre: 128 words each; wsum: 4 words.  bm keeps
// the key bitmap afterwards.  Completion: cp_async_wait_all() then __syncthreads().
__device__ __forceinline__ void stage_lp_team(const VisitOrder& vo, int m, const float* __restrict__ gax,
                                              const float* __restrict__ gay, const float* __restrict__ gb,
                                              float* sX, float* sY, float* sB, unsigned* bm, int* pre,
                                              int* wsum, int tid) {
    const int lane = tid & 31, warp = tid >> 5;
    bm[tid] = 0u;
    __syncthreads();
    for (int q = tid; q < m; q += 128) {
        const uint32_t e = vo.enc(static_cast<uint32_t>(q));
        atomicOr(bm + (e >> 5), 1u << (e & 31u));
    }
    __syncthreads();
    const unsigned w = bm[tid];
    const int incl = warp_inclusive_scan(__popc(w), lane);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int base = 0;
    for (int i = 0; i < warp; ++i) base += wsum[i];
    pre[tid] = base + incl - __popc(w);
    __syncthreads();
    for (int q = tid; q < m; q += 128) {
        const uint32_t e = vo.enc(static_cast<uint32_t>(q));
        const int wi = static_cast<int>(e >> 5);
        stage_copy(kBoxSlots + pre[wi] + __popc(bm[wi] & ((1u << (e & 31u)) - 1u)), q, gax, gay, gb, sX, sY, sB);
    }
}

// The key with rank p in a key bitmap of nwords words (warp-wide; every lane gets it).
__device__ __forceinline__ uint32_t bitmap_select(const unsigned* bm, int nwords, int p, int lane) {
    int base = 0;
    for (int c0 = 0; c0 < nwords; c0 += 32) {
        const unsigned w = (c0 + lane < nwords) ? bm[c0 + lane] : 0u;
        const int c = __popc(w);
        const int incl = warp_inclusive_scan(c, lane);
        const int total = __shfl_sync(kFull, incl, 31);
        if (p < base + total) {
            const unsigned bal = __ballot_sync(kFull, p >= base + incl - c && p < base + incl);
            const int L = __ffs(bal) - 1;
            unsigned wl = __shfl_sync(kFull, w, L);
            const int nth = p - base - __shfl_sync(kFull, incl - c, L);
            for (int i = 0; i < nth; ++i) wl &= wl - 1u;
            return static_cast<uint32_t>((c0 + L) * 32 + __ffs(wl) - 1);
        }
        base += total;
    }
    return 0u;
}

// Constraint id of a stage slot, as reported in out_def: -1 - side for the box,
// otherwise the index of the constraint staged there.
__device__ __forceinline__ int slot_id(int slot, const VisitOrder& vo, const unsigned* bm, int lane) {
    if (slot < kBoxSlots) return -1 - slot;
    const uint64_t dw = vo.domain() >> 5;
    const int nwords = dw > 0 ? static_cast<int>(dw) : 1;
    return static_cast<int>(vo.dec(bitmap_select(bm, nwords, slot - kBoxSlots, lane)));
}

// One lane's share of a 1-D LP: slots j0, j0 + STRIDE, ... below jend.  The line is
// p0 + t u with u oriented so that the objective's end is the right end: the right
// bound (min over den > 0, Eq. 4) is tracked with its slot, the left bound (max over
// den < 0, Eq. 3) by value only.  den is moved off -0 so that a constraint parallel
// to the line (den == 0) yields num / +0: -inf when it excludes the line (num < 0),
// which empties the interval, and +inf or NaN (no effect) when it does not.
// Mixed-precision data of one 1-D LP: the foot of the line in FP64 and the
// near-parallel threshold tau^2 |l|^2 (a work unit with den^2 < lim |g|^2 is
// recomputed in FP64).
struct MixedLine {
    double p0x, p0y;
    float lim;
};

// kFlag: also report (in *np) whether any work unit had near-parallel normals,
// |den| < tau |g| |l| (den^2 < lim |g|^2); kMixed: recompute such work units in FP64
// (the products of the FP32 inputs are exact there).
template <typename Real, int STRIDE, bool kFlag = false, bool kMixed = false>
__device__ __forceinline__ void wu_range(const float* __restrict__ sX, const float* __restrict__ sY,
                                         const float* __restrict__ sB, int j0, int jend, Real p0x, Real p0y,
                                         Real ux, Real uy, Real& thi, int& phi, Real& tlo,
                                         const MixedLine& ml = MixedLine{0.0, 0.0, 0.0f}, bool* np = nullptr) {
    const Real ninf = -real_inf<Real>();
    bool near = false;
#pragma unroll kWuUnroll
    for (int j = j0; j < jend; j += STRIDE) {
        const Real gx = sX[j], gy = sY[j], gb = sB[j];
        Real den = (gx * ux + gy * uy) + Real(0);
        const Real num = gb - (gx * p0x + gy * p0y);
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

// Warp-wide float minimum and maximum (redux.sync on 32-bit floats).
__device__ __forceinline__ float redux_min_f32(float v) {
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;\n" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float redux_max_f32(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;\n" : "=f"(r) : "f"(v));
    return r;
}

// Warp-wide reduction of the 1-D LP state; every lane gets the result: the minimum
// right bound with its lowest slot, the maximum left bound.  FP32 reduces the floats
// directly (redux.sync); FP64 reduces order-preserving 64-bit keys by shuffles.
template <typename Real>
__device__ __forceinline__ void warp_reduce_1dlp(Real& thi, int& phi, Real& tlo) {
    if constexpr (sizeof(Real) == 4) {
        const float m = redux_min_f32(thi);
        phi = __reduce_min_sync(kFull, thi == m ? phi : kNoPos);
        thi = m;
        tlo = redux_max_f32(tlo);
    } else {
        using KT = KeyOf<Real>;
        typename KT::type khi = KT::key(thi), klo = KT::key(tlo);
        warp_min_pair(khi, phi);
        klo = warp_max_key(klo);
        thi = KT::val(khi);
        tlo = KT::val(klo);
    }
}

// Shared-memory protocol between the driving warp and its helpers.
struct TeamJob {
    int cmd;     // kJobRun or kJobDone
    int fslot;   // slots 0 .. fslot-1 take part
    double p0x, p0y, ux, uy;
    float lim;  // near-parallel threshold of the mixed-precision mode
    long long khi[4], klo[4];
    int phi[4];
};
constexpr int kJobRun = 1;
constexpr int kJobDone = 2;
constexpr int kTeamBarJob = 1;   // named barrier: a job (or done) is posted
constexpr int kTeamBarPart = 2;  // named barrier: the helpers' partial results are posted
constexpr int kTeamThreads = 128;
constexpr int kTeamMinSlots = 1024;  // shorter 1-D LPs stay with the driving warp

// Helpers (the CTA's other three warps): wait for jobs until the driver posts kJobDone.
template <typename Real, bool kMixed>
__device__ void team_helper(const float* __restrict__ sX, const float* __restrict__ sY,
                            const float* __restrict__ sB, TeamJob* job, int tid) {
    const int warp = tid >> 5, lane = tid & 31;
    for (;;) {
        named_barrier(kTeamBarJob, kTeamThreads);
        if (job->cmd != kJobRun) break;
        Real thi = real_inf<Real>(), tlo = -real_inf<Real>();
        int phi = kNoPos;
        const MixedLine ml{job->p0x, job->p0y, job->lim};
        wu_range<Real, kTeamThreads, false, kMixed>(sX, sY, sB, tid, job->fslot, static_cast<Real>(job->p0x),
                                             static_cast<Real>(job->p0y), static_cast<Real>(job->ux),
                                             static_cast<Real>(job->uy), thi, phi, tlo, ml);
        using KT = KeyOf<Real>;
        typename KT::type khi = KT::key(thi), klo = KT::key(tlo);
        warp_min_pair(khi, phi);
        klo = warp_max_key(klo);
        if (lane == 0) {
            job->khi[warp] = static_cast<long long>(khi);
            job->klo[warp] = static_cast<long long>(klo);
            job->phi[warp] = phi;
        }
        named_barrier(kTeamBarPart, kTeamThreads);
    }
}

// Seidel iterations of one staged LP by one warp (lane = 0..31).  With a team
// (kTeam, job != nullptr), 1-D LPs over at least kTeamMinSlots slots are shared with
// the helper warps, and the driver posts kJobDone when it has finished; without one
// (job unused) the team code is compiled out.  Writes the LP's outputs.
template <typename Real, bool kMixed, bool kTeam>
__device__ void drive_lp(const Params& P, int64_t lp, int m, float cxf, float cyf, const VisitOrder& vo,
                         const float* __restrict__ sX, const float* __restrict__ sY,
                         const float* __restrict__ sB, const unsigned* bm, int lane, TeamJob* job) {
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
    int k = 0;
    // With a team (large LPs, long violation-free stretches) the values of positions
    // k + lane are loaded one step ahead of their test, so that the shared-memory
    // latency leaves the critical path of the scan.
    float fx = 0.0f, fy = 0.0f, fb = 0.0f;
    if (kTeam && lane < m) {
        fx = sX[kBoxSlots + lane];
        fy = sY[kBoxSlots + lane];
        fb = sB[kBoxSlots + lane];
    }
    while (k < m) {
        const int p = k + lane;
        float nx = 0.0f, ny = 0.0f, nb = 0.0f;
        if constexpr (kTeam) {
            if (p + 32 < m) {
                nx = sX[kBoxSlots + p + 32];
                ny = sY[kBoxSlots + p + 32];
                nb = sB[kBoxSlots + p + 32];
            }
        } else if (p < m) {
            fx = sX[kBoxSlots + p];
            fy = sY[kBoxSlots + p];
            fb = sB[kBoxSlots + p];
        }
        bool viol = false;
        if (p < m) {
            fin = fmaf(fx, 0.0f, fmaf(fy, 0.0f, fmaf(fb, 0.0f, fin)));
            const Real gx = fx, gy = fy, gb = fb;
            const Real s = gx * vx + gy * vy - gb;
            const Real tol = eps * (real_abs(gx) * avx + real_abs(gy) * avy + real_abs(gb));
            viol = s > tol;
        }
        const unsigned bal = __ballot_sync(kFull, viol);
        const int first = bal ? k + __ffs(bal) - 1 : kNoPos;
        if (first == kNoPos) {
            k += 32;
            if constexpr (kTeam) {
                fx = nx;
                fy = ny;
                fb = nb;
            }
            continue;
        }
        const int fslot = kBoxSlots + first;
        k = first + 1;
        // ---- 1-D LP on the violated line l: lx*x + ly*y = lb
        const Real lx = sX[fslot], ly = sY[fslot], lb = sB[fslot];
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
        if (kTeam && fslot >= kTeamMinSlots) {
            if constexpr (kMixed) foot64();
            if (lane == 0) {
                job->cmd = kJobRun;
                job->fslot = fslot;
                job->p0x = kMixed ? ml.p0x : static_cast<double>(p0x);
                job->p0y = kMixed ? ml.p0y : static_cast<double>(p0y);
                job->ux = static_cast<double>(ux);
                job->uy = static_cast<double>(uy);
                job->lim = ml.lim;
            }
            named_barrier(kTeamBarJob, kTeamThreads);
            // the driver takes the slots of its own thread index, like every helper
            wu_range<Real, kTeamThreads, false, kMixed>(sX, sY, sB, static_cast<int>(threadIdx.x), fslot, p0x, p0y,
                                                        ux, uy, thi, phi, tlo, ml);
            warp_reduce_1dlp<Real>(thi, phi, tlo);
            named_barrier(kTeamBarPart, kTeamThreads);
            using KT = KeyOf<Real>;
            typename KT::type khi = KT::key(thi), klo = KT::key(tlo);
            const int self = static_cast<int>(threadIdx.x >> 5);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (w == self) continue;
                const auto kh = static_cast<typename KT::type>(job->khi[w]);
                const int ph = job->phi[w];
                if (kh < khi || (kh == khi && ph < phi)) { khi = kh; phi = ph; }
                const auto kl = static_cast<typename KT::type>(job->klo[w]);
                klo = kl > klo ? kl : klo;
            }
            thi = KT::val(khi);
            tlo = KT::val(klo);
        } else if (!kMixed && fslot <= 32) {
            // a short 1-D LP: one slot per lane, no loop
            if (lane < fslot) {
                const Real gx = sX[lane], gy = sY[lane], gb = sB[lane];
                const Real den = (gx * ux + gy * uy) + Real(0);
                const Real num = gb - (gx * p0x + gy * p0y);
                const Real t = real_div<Real>(num, den);
                const bool right = den >= Real(0);
                if (right && t < thi) { thi = t; phi = lane; }
                tlo = right ? tlo : t;
            }
            warp_reduce_1dlp<Real>(thi, phi, tlo);
        } else if (!kMixed && fslot <= 64) {
            // a short 1-D LP: at most two slots per lane, no loop
            const Real ninf = -real_inf<Real>();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                if (j < fslot) {
                    const Real gx = sX[j], gy = sY[j], gb = sB[j];
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
            warp_reduce_1dlp<Real>(thi, phi, tlo);
        } else {
            bool np = false;
            wu_range<Real, 32, kMixed>(sX, sY, sB, lane, fslot, p0x, p0y, ux, uy, thi, phi, tlo, ml, &np);
            if (kMixed && __any_sync(kFull, np)) {
                // a near-parallel pair: redo this 1-D LP with FP64 intersections for them
                foot64();
                thi = real_inf<Real>();
                tlo = -real_inf<Real>();
                phi = kNoPos;
                wu_range<Real, 32, false, kMixed>(sX, sY, sB, lane, fslot, p0x, p0y, ux, uy, thi, phi, tlo, ml);
            }
            warp_reduce_1dlp<Real>(thi, phi, tlo);
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
                wu_range<double, 32>(sX, sY, sB, lane, fslot, ml.p0x, ml.p0y, static_cast<double>(ux),
                                     static_cast<double>(uy), th64, ph64, tl64);
                warp_reduce_1dlp<double>(th64, ph64, tl64);
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
        if (kTeam && k + lane < m) {
            fx = sX[kBoxSlots + k + lane];
            fy = sY[kBoxSlots + k + lane];
            fb = sB[kBoxSlots + k + lane];
        }
    }
    // positions never scanned (the LP stopped early) still take part in the finiteness check
    if (P.check_finite) {
        for (int p = k + lane; p < m; p += 32)
            fin = fmaf(sX[kBoxSlots + p], 0.0f, fmaf(sY[kBoxSlots + p], 0.0f, fmaf(sB[kBoxSlots + p], 0.0f, fin)));
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

}  // namespace lp2d
