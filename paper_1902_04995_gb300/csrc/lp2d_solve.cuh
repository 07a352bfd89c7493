// lp2d_solve.cuh -- one LP solved by a team of W warps (W = 1: a single warp).
//
// The LP's constraints are staged once from HBM (coalesced, in stored order) into
// shared memory at their visit positions pi^{-1}(q), so that every later read --
// the violation scan and every 1-D LP -- is a contiguous shared-memory read in visit
// order (the paper stages the current line and the per-LP results in shared memory,
// Sec. 3; here the whole LP is staged, since it is re-read by every 1-D LP).
//
// Control flow follows serial Seidel exactly (Sec. 2.1):
//   * scan: the team tests T = 32 W consecutive visit positions k..k+T-1 against the
//     current optimum v at once and takes the first violated one (ballot).  Every
//     position before it is satisfied by v, so serial Seidel would have left v
//     unchanged there: the trajectory is the serial one.
//   * 1-D LP on the violated line l (p0 + t u): every earlier constraint h (box sides
//     at positions -4..-1, then positions 0..k-1) gives sigma = num/den; den > 0 bounds
//     t from the right (Eq. 4, min), den < 0 from the left (Eq. 3, max), den == 0 with
//     num < 0 excludes the line.  Each lane reduces its strided share, then the warp
//     (redux.sync on order-preserving integer keys) and the team (shared memory)
//     reduce (value, position) pairs, ties going to the earliest position.
//   * empty interval (left > right) or an excluding parallel constraint: infeasible.
//     Otherwise t* = right end if c.u > 0, else left end.
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

template <int W>
__device__ __forceinline__ void team_sync() {
    if constexpr (W == 1) __syncwarp();
    else __syncthreads();
}

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

// Team-wide minimum of an int (first violated visit position).
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

// Team-wide reduction of a 1-D LP: (min right key, its position), (max left key,
// its position), OR of the parallel-exclusion flag.
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

// Constraint at visit position p: from the shared-memory stage, or (for LPs larger
// than the stage) straight from global memory through pi.
template <bool kStaged>
struct ConstraintSource {
    const float* __restrict__ X;
    const float* __restrict__ Y;
    const float* __restrict__ B;
    const VisitOrder* vo;

    template <typename Real>
    __device__ __forceinline__ void get(int p, Real& gx, Real& gy, Real& gb, bool& werr) const {
        if constexpr (kStaged) {
            gx = static_cast<Real>(X[p]);
            gy = static_cast<Real>(Y[p]);
            gb = static_cast<Real>(B[p]);
        } else {
            const uint32_t q = vo->fwd(static_cast<uint32_t>(p), werr);
            gx = static_cast<Real>(__ldg(X + q));
            gy = static_cast<Real>(__ldg(Y + q));
            gb = static_cast<Real>(__ldg(B + q));
        }
    }
};

// Solve LP `lp` (constraints base .. base+m-1) with a team of W warps; `tid` is the
// thread's index within the team.  kStaged: stage into sX/sY/sB (capacity >= m);
// otherwise read through pi from global memory.  Writes the LP's outputs.
template <int W, typename Real, bool kStaged>
__device__ void solve_lp(const Params& P, int64_t lp, int64_t base, int m,
                         float* __restrict__ sX, float* __restrict__ sY, float* __restrict__ sB,
                         TeamScratch<W>* sc, unsigned& phase, int tid) {
    constexpr int T = 32 * W;
    using KT = KeyOf<Real>;
    using K = typename KT::type;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    VisitOrder vo;
    vo.init(P.seed + static_cast<uint64_t>(lp), static_cast<uint32_t>(m));
    bool werr = false;
    const float cxf = __ldg(P.obj + 2 * lp);
    const float cyf = __ldg(P.obj + 2 * lp + 1);
    const Real cx = static_cast<Real>(cxf), cy = static_cast<Real>(cyf);

    // ---- staging: coalesced loads in stored order, scattered to visit positions.
    float fin = 0.0f;  // becomes NaN iff some input is NaN or +-Inf
    if constexpr (kStaged) {
        const float* __restrict__ gax = P.ax + base;
        const float* __restrict__ gay = P.ay + base;
        const float* __restrict__ gb = P.b + base;
        for (int q0 = tid; q0 < m; q0 += 4 * T) {
            float x[4], y[4], z[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + u * T;
                x[u] = y[u] = z[u] = 0.0f;
                if (q < m) {
                    x[u] = __ldcs(gax + q);
                    y[u] = __ldcs(gay + q);
                    z[u] = __ldcs(gb + q);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int q = q0 + u * T;
                if (q < m) {
                    const uint32_t p = vo.inv(static_cast<uint32_t>(q), werr);
                    sX[p] = x[u];
                    sY[p] = y[u];
                    sB[p] = z[u];
                    fin = fmaf(x[u], 0.0f, fin);
                    fin = fmaf(y[u], 0.0f, fin);
                    fin = fmaf(z[u], 0.0f, fin);
                }
            }
        }
    } else {
        if (P.check_finite) {
            for (int q = tid; q < m; q += T) {
                fin = fmaf(__ldg(P.ax + base + q), 0.0f, fin);
                fin = fmaf(__ldg(P.ay + base + q), 0.0f, fin);
                fin = fmaf(__ldg(P.b + base + q), 0.0f, fin);
            }
        }
    }
    if (W == 1) __syncwarp();
    bool bad = team_any<W>(P.check_finite && (fin != fin), sc, phase, warp, lane);  // also the stage barrier
    bad = bad || !(fabsf(cxf) <= 3.402823466e38f) || !(fabsf(cyf) <= 3.402823466e38f);

    const ConstraintSource<kStaged> src{kStaged ? sX : P.ax + base, kStaged ? sY : P.ay + base,
                                        kStaged ? sB : P.b + base, &vo};

    // ---- Seidel iterations.  Start at the box corner maximising c.
    Real vx = (cx >= Real(0)) ? Real(P.xmax) : Real(P.xmin);
    Real vy = (cy >= Real(0)) ? Real(P.ymax) : Real(P.ymin);
    int d0 = (cx >= Real(0)) ? -4 : -3;  // visit positions of the defining pair
    int d1 = (cy >= Real(0)) ? -2 : -1;
    int status = bad ? kBadInput : -1;
    int nviol = 0;
    const Real eps = (sizeof(Real) == 4) ? Real(P.eps32) : Real(P.eps64);

    int k = 0;
    while (!bad && k < m) {
        // scan T positions for the first violated one
        const int p = k + tid;
        bool viol = false;
        if (p < m) {
            Real gx, gy, gb;
            src.get(p, gx, gy, gb, werr);
            const Real s = gx * vx + gy * vy - gb;
            const Real tol = eps * (real_abs(gx * vx) + real_abs(gy * vy) + real_abs(gb));
            viol = s > tol;
        }
        const unsigned bal = __ballot_sync(kFull, viol);
        const int wfirst = bal ? (k + warp * 32 + __ffs(bal) - 1) : kNoPos;
        const int first = team_min<W>(wfirst, sc, phase, warp, lane);
        if (first == kNoPos) {
            k += T;
            continue;
        }
        // ---- 1-D LP on the violated line l: lx*x + ly*y = lb
        Real lx, ly, lb;
        src.get(first, lx, ly, lb, werr);
        const Real nrm2 = lx * lx + ly * ly;
        if (nrm2 == Real(0)) {  // 0.x <= lb < 0
            status = kInfeasible;
            d0 = first;
            break;
        }
        const Real sc0 = lb / nrm2;
        const Real p0x = lx * sc0, p0y = ly * sc0;  // foot of l
        const Real ux = -ly, uy = lx;              // direction of l
        Real thi = real_inf<Real>(), tlo = -real_inf<Real>();
        int phi = kNoPos, plo = kNoPos;
        bool par = false;
        if (tid < 4) {
            Real gx, gy, gb;
            box_side<Real>(P, tid, gx, gy, gb);
            const Real den = gx * ux + gy * uy;
            const Real num = gb - (gx * p0x + gy * p0y);
            const Real t = real_div<Real>(num, den);
            if (den > Real(0)) { thi = t; phi = tid - 4; }
            else if (den < Real(0)) { tlo = t; plo = tid - 4; }
            else if (num < Real(0)) par = true;
        }
        for (int j = tid; j < first; j += T) {
            Real gx, gy, gb;
            src.get(j, gx, gy, gb, werr);
            const Real den = gx * ux + gy * uy;
            const Real num = gb - (gx * p0x + gy * p0y);
            const Real t = real_div<Real>(num, den);
            if (den > Real(0)) {
                if (t < thi) { thi = t; phi = j; }
            } else if (den < Real(0)) {
                if (t > tlo) { tlo = t; plo = j; }
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
            d0 = first;
            break;
        }
        const Real cu = cx * ux + cy * uy;
        const bool right = cu > Real(0);
        const Real t = right ? thi : tlo;
        vx = p0x + t * ux;
        vy = p0y + t * uy;
        d0 = first;
        d1 = right ? phi : plo;
        k = first + 1;
    }

    if (werr && P.ws) atomicOr(P.ws + kWsError, static_cast<unsigned long long>(kDevErrWalkLimit));
    if (tid == 0) {
        if (status < 0) status = (d0 < 0 || d1 < 0) ? kBoxBounded : kOptimal;
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
            bool e2 = false;
            P.out_def[2 * lp] = def_id(d0, vo, e2);
            P.out_def[2 * lp + 1] = def_id(d1, vo, e2);
        }
    }
}

}  // namespace lp2d
