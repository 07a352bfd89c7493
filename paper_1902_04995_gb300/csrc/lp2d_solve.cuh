// lp2d_solve.cuh -- one LP too large for the shared-memory stage, solved by a team of
// W warps reading its constraints from global memory (L1/L2 hold the LP after the
// first touch).
//
// Visit order without a stage: scanning the key domain of the Feistel permutation
// upward and skipping keys whose constraint index is >= m lists the constraints in
// visit order (increasing key), so "the constraints before position k" are "the
// constraints whose key is below the key of k".  The team scans T = 32 W keys at a
// time; the first violated one (ballot) is the next step of serial Seidel (Sec. 2.1).
// Its 1-D LP runs over the box sides (tags 0..3) and every valid key below it
// (tag 4 + key): den > 0 bounds t from the right (Eq. 4, min), den < 0 from the left
// (Eq. 3, max), den == 0 with num < 0 excludes the line; ties go to the lowest tag,
// the earliest constraint.
#pragma once

#include "lp2d_device.cuh"

namespace lp2d {

// Shared-memory scratch for the reductions of a team of W > 1 warps.  Double
// buffered by a phase bit, so one barrier per reduction suffices.
template <int W>
struct TeamScratch {
    long long khi[2][W];
    long long klo[2][W];
    int phi[2][W];
    int plo[2][W];
    int flag[2][W];
};

// Team-wide OR of a predicate.
template <int W>
__device__ __forceinline__ bool team_any(bool v, TeamScratch<W>* sc, unsigned& phase, int warp, int lane) {
    bool w = __any_sync(kFull, v);
    if constexpr (W == 1) {
        return w;
    } else {
        const int s = phase & 1u;
        ++phase;
        if (lane == 0) sc->flag[s][warp] = w ? 1 : 0;
        __syncthreads();
        int r = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) r |= sc->flag[s][i];
        return r != 0;
    }
}

// Team-wide minimum of an int.
template <int W>
__device__ __forceinline__ int team_min(int v, TeamScratch<W>* sc, unsigned& phase, int warp, int lane) {
    int w = __reduce_min_sync(kFull, v);
    if constexpr (W == 1) {
        return w;
    } else {
        const int s = phase & 1u;
        ++phase;
        if (lane == 0) sc->phi[s][warp] = w;
        __syncthreads();
        int r = sc->phi[s][0];
#pragma unroll
        for (int i = 1; i < W; ++i) r = min(r, sc->phi[s][i]);
        return r;
    }
}

// Team-wide reduction of a 1-D LP: (min right key, its tag), (max left key, its
// tag), OR of the parallel-exclusion flag.
template <int W, typename K>
__device__ __forceinline__ void team_reduce_1dlp(K& khi, int& phi, K& klo, int& plo, bool& par,
                                                 TeamScratch<W>* sc, unsigned& phase, int warp, int lane) {
    warp_min_pair(khi, phi);
    warp_max_pair(klo, plo);
    par = __any_sync(kFull, par);
    if constexpr (W > 1) {
        const int s = phase & 1u;
        ++phase;
        if (lane == 0) {
            sc->khi[s][warp] = static_cast<long long>(khi);
            sc->phi[s][warp] = phi;
            sc->klo[s][warp] = static_cast<long long>(klo);
            sc->plo[s][warp] = plo;
            sc->flag[s][warp] = par ? 1 : 0;
        }
        __syncthreads();
        khi = static_cast<K>(sc->khi[s][0]);
        phi = sc->phi[s][0];
        klo = static_cast<K>(sc->klo[s][0]);
        plo = sc->plo[s][0];
        int f = sc->flag[s][0];
#pragma unroll
        for (int i = 1; i < W; ++i) {
            const K kh = static_cast<K>(sc->khi[s][i]);
            const int ph = sc->phi[s][i];
            if (kh < khi || (kh == khi && ph < phi)) { khi = kh; phi = ph; }
            const K kl = static_cast<K>(sc->klo[s][i]);
            const int pl = sc->plo[s][i];
            if (kl > klo || (kl == klo && pl < plo)) { klo = kl; plo = pl; }
            f |= sc->flag[s][i];
        }
        par = f != 0;
    }
}

// Largest LP the key-domain path takes: its tags (4 + key) must fit an int.
constexpr int64_t kMaxKeyPathM = 1ll << 30;

// Solve LP `lp` (constraints base .. base+m-1, m <= kMaxKeyPathM) with a team of W
// warps reading global memory; `tid` is the thread's index within the team.
// Writes the LP's outputs.
template <int W, typename Real, bool kMixed = false>
__device__ void solve_lp_keys(const Params& P, int64_t lp, int64_t base, int m, TeamScratch<W>* sc,
                              unsigned& phase, int tid) {
    constexpr int T = 32 * W;
    using KT = KeyOf<Real>;
    using K = typename KT::type;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const float* __restrict__ gax = P.ax + base;
    const float* __restrict__ gay = P.ay + base;
    const float* __restrict__ gbb = P.b + base;

    VisitOrder vo;
    vo.init(P.seed + static_cast<uint64_t>(lp), static_cast<uint32_t>(m));
    const uint32_t dom = static_cast<uint32_t>(vo.domain());  // <= 2^30
    const float cxf = __ldg(P.obj + 2 * lp);
    const float cyf = __ldg(P.obj + 2 * lp + 1);
    const Real cx = static_cast<Real>(cxf), cy = static_cast<Real>(cyf);

    float fin = 0.0f;
    if (P.check_finite) {
        for (int q = tid; q < m; q += T)
            fin = fmaf(__ldg(gax + q), 0.0f, fmaf(__ldg(gay + q), 0.0f, fmaf(__ldg(gbb + q), 0.0f, fin)));
    }
    bool bad = team_any<W>(fin != fin, sc, phase, warp, lane);
    bad = bad || !(fabsf(cxf) <= 3.402823466e38f) || !(fabsf(cyf) <= 3.402823466e38f);

    Real vx = (cx >= Real(0)) ? Real(P.xmax) : Real(P.xmin);
    Real vy = (cy >= Real(0)) ? Real(P.ymax) : Real(P.ymin);
    int d0 = (cx >= Real(0)) ? 0 : 1;  // tags of the defining pair (box sides 0..3)
    int d1 = (cy >= Real(0)) ? 2 : 3;
    int status = bad ? kBadInput : -1;
    int nviol = 0;
    const Real eps = (sizeof(Real) == 4) ? Real(P.eps32) : Real(P.eps64);

    uint32_t e0 = 0;  // next key to scan
    while (!bad && e0 < dom) {
        const uint32_t e = e0 + static_cast<uint32_t>(tid);
        bool viol = false;
        if (e < dom) {
            const uint32_t q = vo.dec(e);
            if (q < static_cast<uint32_t>(m)) {
                const Real gx = __ldg(gax + q), gy = __ldg(gay + q), gb = __ldg(gbb + q);
                const Real s = gx * vx + gy * vy - gb;
                const Real tol = eps * (real_abs(gx * vx) + real_abs(gy * vy) + real_abs(gb));
                viol = s > tol;
            }
        }
        const unsigned bal = __ballot_sync(kFull, viol);
        const int wfirst = bal ? static_cast<int>(e0) + warp * 32 + __ffs(bal) - 1 : kNoPos;
        const int first = team_min<W>(wfirst, sc, phase, warp, lane);
        if (first == kNoPos) {
            e0 += T;
            continue;
        }
        const uint32_t lq = vo.dec(static_cast<uint32_t>(first));
        const Real lx = __ldg(gax + lq), ly = __ldg(gay + lq), lb = __ldg(gbb + lq);
        const Real nrm2 = lx * lx + ly * ly;
        if (nrm2 == Real(0)) {
            status = kInfeasible;
            break;
        }
        const Real sc0 = lb / nrm2;
        const Real p0x = lx * sc0, p0y = ly * sc0;
        const Real ux = -ly, uy = lx;
        // mixed precision: FP64 foot of the line and the near-parallel threshold
        double p0x64 = 0.0, p0y64 = 0.0;
        float lim = 0.0f;
        if constexpr (kMixed) {
            const double lx64 = lx, ly64 = ly, sc64 = static_cast<double>(lb) / (lx64 * lx64 + ly64 * ly64);
            p0x64 = lx64 * sc64;
            p0y64 = ly64 * sc64;
            lim = P.tau * P.tau * static_cast<float>(nrm2);
        }
        Real thi = real_inf<Real>(), tlo = -real_inf<Real>();
        int phi = kNoPos, plo = kNoPos;
        bool par = false;
        if (tid < 4) {
            const Real gx = (tid == 0) ? Real(1) : (tid == 1) ? Real(-1) : Real(0);
            const Real gy = (tid == 2) ? Real(1) : (tid == 3) ? Real(-1) : Real(0);
            const Real gb = (tid == 0) ? Real(P.xmax) : (tid == 1) ? Real(-P.xmin) : (tid == 2) ? Real(P.ymax)
                                                                                                : Real(-P.ymin);
            const Real den = gx * ux + gy * uy;
            const Real num = gb - (gx * p0x + gy * p0y);
            const Real t = real_div<Real>(num, den);
            if (den > Real(0)) { thi = t; phi = tid; }
            else if (den < Real(0)) { tlo = t; plo = tid; }
            else if (num < Real(0)) par = true;
        }
        for (int ek = tid; ek < first; ek += T) {
            const uint32_t g = vo.dec(static_cast<uint32_t>(ek));
            if (g >= static_cast<uint32_t>(m)) continue;
            const Real gx = __ldg(gax + g), gy = __ldg(gay + g), gb = __ldg(gbb + g);
            Real den = gx * ux + gy * uy;
            Real num = gb - (gx * p0x + gy * p0y);
            Real t = real_div<Real>(num, den);
            if constexpr (kMixed) {
                if (den * den < lim * (gx * gx + gy * gy)) {  // near-parallel: redo in FP64
                    const double d64 = (static_cast<double>(gx) * static_cast<double>(ux) +
                                        static_cast<double>(gy) * static_cast<double>(uy)) + 0.0;
                    const double n64 = static_cast<double>(gb) -
                                       (static_cast<double>(gx) * p0x64 + static_cast<double>(gy) * p0y64);
                    t = static_cast<Real>(n64 / d64);
                    den = (d64 > 0.0) ? Real(1) : (d64 < 0.0) ? Real(-1) : Real(0);
                    num = static_cast<Real>(n64);
                }
            }
            if (den > Real(0)) {
                if (t < thi) { thi = t; phi = 4 + ek; }
            } else if (den < Real(0)) {
                if (t > tlo) { tlo = t; plo = 4 + ek; }
            } else if (num < Real(0)) {
                par = true;
            }
        }
        K khi = KT::key(thi), klo = KT::key(tlo);
        team_reduce_1dlp<W, K>(khi, phi, klo, plo, par, sc, phase, warp, lane);
        ++nviol;
        thi = KT::val(khi);
        tlo = KT::val(klo);
        if (par || tlo > thi) {
            status = kInfeasible;
            break;
        }
        const Real cu = cx * ux + cy * uy;
        const bool right = cu > Real(0);
        const Real t = right ? thi : tlo;
        vx = p0x + t * ux;
        vy = p0y + t * uy;
        d0 = 4 + first;
        d1 = right ? phi : plo;
        e0 = static_cast<uint32_t>(first) + 1u;
    }

    if (tid == 0) {
        if (status < 0) status = (d0 < 4 || d1 < 4) ? kBoxBounded : kOptimal;
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
            P.out_def[2 * lp] = d0 < 4 ? -1 - d0 : static_cast<int>(vo.dec(static_cast<uint32_t>(d0 - 4)));
            P.out_def[2 * lp + 1] = d1 < 4 ? -1 - d1 : static_cast<int>(vo.dec(static_cast<uint32_t>(d1 - 4)));
        }
    }
}

}  // namespace lp2d
