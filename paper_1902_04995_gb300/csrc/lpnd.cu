// lpnd.cu -- the batched d-dimensional Seidel solver (d = 2..5) and its extern "C" entry.
//
// Seidel's method (Sec. 2.1 gives it in 2-D; Sec. 6 names higher dimensions) as a
// recursion over affine subspaces x = p + sum_i s_i E_i of R^d.  One warp solves one
// LP staged in shared memory in visit order: slots 0..2d-1 hold the box planes
// (x_0 <= max_0, -x_0 <= -min_0, x_1 <= max_1, ...), slot 2d + p the constraint
// visited at p; coefficient t of a slot sits in array t of the stage, b in array d.
//   - every level scans 32 slots per step against the current point in R^d (the
//     2-D solver's relative tolerance); the first violated one is the next step of
//     serial Seidel;
//   - a violation of constraint g inside a k-dimensional subspace moves the point
//     onto g's hyperplane: the (k-1)-dimensional frame is one pivoted elimination
//     step (A_i = g.E_i, r = b - g.p, J = argmax |A_J|, p' = p + (r/A_J) E_J,
//     E'_i = E_i - (A_i/A_J) E_J, each quotient as a product with 1/A_J), kept in
//     the warp's slice of shared memory, and
//     the LP on it runs over the box and every earlier slot;
//   - a sub-LP of dimension k >= 2 starts at the best vertex of the box inside its
//     subspace: one candidate per lane (k distinct axes and a side of each, C(d,k) 2^k
//     of them), a k x k solve with partial pivoting, the other axes checked against
//     the box, a warp arg-max of c.x;
//   - dimension 1 is the 1-D LP of Eqs. 3 and 4 with the 2-D solver's rules (lanes
//     reduce strided slots, redux.sync combines them); an infeasible sub-LP makes the
//     LP infeasible.
// A persistent grid of 4-warp CTAs pulls LPs from two queues: LPs of more than
// 512 - 2d constraints go to warps 0 and 1 with half of the CTA's stage each, smaller
// ones to all four warps with a quarter each.  LPs above 1024 - 2d are BAD_INPUT.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "lpnd.h"
#include "lp2d_internal.h"
#include "lp2d_staged.cuh"
#include "lp_stage_big.cuh"

namespace lp2d {

constexpr int kWarpsN = 4;
constexpr int kQuarterN = 512;           // stage slots of a warp in the small-LP phase
constexpr int kHalfN = 1024;             // stage slots of a warp in the mid-size phase
constexpr int kStageN = 4 * kQuarterN;   // slots per array of a CTA's stage
constexpr unsigned kDevErrTooLargeN = 4u;

struct ParamsN {
    const float* a[LPND_MAX_DIM];
    const float* __restrict__ b;
    const int64_t* __restrict__ offsets;
    int64_t n_lp;
    const float* __restrict__ obj;
    float box[2 * LPND_MAX_DIM];
    uint64_t seed;
    void* out_x;
    int32_t* out_status;
    int32_t* out_nviol;
    int32_t* out_def;
    unsigned long long* ws;
    float eps32;
    double eps64;
    int chunk;
    int check_finite;
};

__host__ __device__ constexpr int binom(int n, int k) {
    return (k < 0 || k > n) ? 0 : (k == 0 || k == n) ? 1 : binom(n - 1, k - 1) + binom(n - 1, k);
}

// Frames of levels 1..D-1 in a warp's frame area: level k holds p and E_0..E_{k-1},
// D values each, from offset D (k (k+1)/2 - 1).
template <int D> __host__ __device__ constexpr int frame_off(int k) { return D * (k * (k + 1) / 2 - 1); }
template <int D> constexpr int kFrameReals = frame_off<D>(D);

template <int D, typename Real> constexpr size_t smem_bytes_n() {
    return sizeof(float) * (D + 1) * kStageN + sizeof(Real) * kWarpsN * kFrameReals<D> +
           sizeof(int) * kWarpsN * D + sizeof(unsigned) * kWarpsN * 32;
}

// Resident CTAs per SM that shared memory allows (228 KB per SM, 1 KB reserved per
// CTA): the register budget FP32 is compiled for.  FP64 (a small fraction of the
// FP32 rate on this part) takes half of it and keeps its wider state in registers.
template <int D, typename Real> constexpr int min_ctas_n() {
    return static_cast<int>(233472 / (smem_bytes_n<D, Real>() + 1024)) / (sizeof(Real) == 4 ? 1 : 2);
}

// One warp's view of the LP it solves.  x and c are uniform across the warp.
template <typename Real, int D, int S = kStageN>
struct WarpN {
    static constexpr int kS = S;  // slots per array of the stage
    const float* s;  // coefficient t of slot i at s[t * S + i], b at s[D * S + i]
    Real* fr;        // frames of levels 1..D-1
    int* defs;       // slots of the D constraints through x; level k owns defs[D-k .. D-1]
    Real c[D];
    Real x[D];
    Real eps;
    int lane;
    int nviol;
};

template <typename Real, int D, int S>
__device__ __forceinline__ bool violates_n(const float* s, int sl, const Real (&x)[D], Real eps) {
    const Real gb = s[D * S + sl];
    Real acc = -gb, tol = real_abs(gb);
#pragma unroll
    for (int t = 0; t < D; ++t) {
        const Real pr = Real(s[t * S + sl]) * x[t];
        acc += pr;
        tol += real_abs(pr);
    }
    return acc > eps * tol;
}

// 1 / v rounded to nearest (one reciprocal per pivot instead of a division per use).
__device__ __forceinline__ float real_rcp(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double real_rcp(double v) { return __drcp_rn(v); }

// M y = R for a K x K system, partial pivoting by conditional row swaps (every index
// known at compile time, so M stays in registers); false if a pivot is zero.  M's
// diagonal is overwritten with the pivots' reciprocals.
template <typename Real, int K>
__device__ __forceinline__ bool gauss_solve(Real (&M)[K][K], Real (&R)[K], Real (&y)[K]) {
#pragma unroll
    for (int col = 0; col < K; ++col) {
#pragma unroll
        for (int r = col + 1; r < K; ++r) {
            const bool sw = real_abs(M[r][col]) > real_abs(M[col][col]);
#pragma unroll
            for (int j = col; j < K; ++j) {
                const Real u = M[col][j], v = M[r][j];
                M[col][j] = sw ? v : u;
                M[r][j] = sw ? u : v;
            }
            const Real u = R[col], v = R[r];
            R[col] = sw ? v : u;
            R[r] = sw ? u : v;
        }
        if (!(M[col][col] != Real(0))) return false;
        M[col][col] = real_rcp(M[col][col]);  // the pivot's reciprocal from here on
#pragma unroll
        for (int r = col + 1; r < K; ++r) {
            const Real f = M[r][col] * M[col][col];
#pragma unroll
            for (int j = col + 1; j < K; ++j) M[r][j] -= f * M[col][j];
            R[r] -= f * R[col];
        }
    }
#pragma unroll
    for (int i = K - 1; i >= 0; --i) {
        Real v = R[i];
#pragma unroll
        for (int j = i + 1; j < K; ++j) v -= M[i][j] * y[j];
        y[i] = v * M[i][i];
    }
    return true;
}

// The rank-th subset of K axes out of D, as a bit mask, in increasing mask order.
__host__ __device__ constexpr unsigned mask_of(int D, int K, int rank) {
    int seen = 0;
    for (unsigned mk = 0; mk < (1u << D); ++mk) {
        int bits = 0;
        for (unsigned v = mk; v != 0u; v &= v - 1u) ++bits;
        if (bits == K) {
            if (seen == rank) return mk;
            ++seen;
        }
    }
    return 0u;
}

// The same for a rank known only at run time: a select over the C(D, K) constants.
template <int D, int K>
__device__ __forceinline__ unsigned nth_mask(int rank) {
    unsigned found = mask_of(D, K, 0);
#pragma unroll
    for (int r = 1; r < binom(D, K); ++r) found = (rank == r) ? mask_of(D, K, r) : found;
    return found;
}

// Start of a sub-LP on the level-K frame (2 <= K < D): the best vertex of the box in
// the subspace.  Sets x and defs[D-K .. D-1]; false if the subspace misses the box.
template <typename Real, int D, int K, typename WT>
__device__ __forceinline__ bool box_start(WT& W) {
    using KT = KeyOf<Real>;
    constexpr int S = WT::kS;
    constexpr int kCands = binom(D, K) << K;
    const Real* F = W.fr + frame_off<D>(K);
    const float* sb = W.s + D * S;  // slot 2a: b = max_a; slot 2a + 1: b = -min_a
    bool found = false;
    Real best = Real(0);
    unsigned best_mask = 0u;
    int best_sg = 0, best_lex = 0;
#pragma unroll 1
    for (int q0 = 0; q0 < kCands; q0 += 32) {
        const int q = q0 + W.lane;
        bool ok = false;
        Real val = Real(0), xc[D];
        unsigned mask = 0u;
        const int sg = q & ((1 << K) - 1);
        int lex = 0;  // the candidate's box planes 2a + side, in increasing order, as digits base 2D
#pragma unroll
        for (int t = 0; t < D; ++t) xc[t] = Real(0);
        if (q < kCands) {
            mask = nth_mask<D, K>(q >> K);
            Real M[K][K], R[K], y[K];
            unsigned mk = mask;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                const int a = __ffs(mk) - 1;
                mk &= mk - 1u;
                lex = lex * (2 * D) + 2 * a + ((sg >> r) & 1);
                const Real v = ((sg >> r) & 1) ? -Real(sb[2 * a + 1]) : Real(sb[2 * a]);
                R[r] = v - F[a];
#pragma unroll
                for (int i = 0; i < K; ++i) M[r][i] = F[D * (1 + i) + a];
            }
            if (gauss_solve<Real, K>(M, R, y)) {
                ok = true;
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    Real v = F[t];
#pragma unroll
                    for (int i = 0; i < K; ++i) v += y[i] * F[D * (1 + i) + t];
                    xc[t] = v;
                    if (!((mask >> t) & 1u)) {
                        const Real hi = sb[2 * t], lo = -Real(sb[2 * t + 1]);
                        if (v - hi > W.eps * (real_abs(v) + real_abs(hi))) ok = false;
                        if (lo - v > W.eps * (real_abs(v) + real_abs(lo))) ok = false;
                    }
                    val += W.c[t] * v;
                }
            }
        }
        // the largest value; on ties the candidate whose box planes come first in
        // lexicographic order (R24), as the oracle enumerates them
        const typename KT::type key = ok ? KT::key(val) : KT::key(-real_inf<Real>());
        const typename KT::type kmax = warp_max_key(key);
        const int lmin = __reduce_min_sync(kFull, (ok && key == kmax) ? lex : INT_MAX);
        const unsigned hit = __ballot_sync(kFull, ok && key == kmax && lex == lmin);
        const int who = hit != 0u ? __ffs(hit) - 1 : kNoPos;
        if (who != kNoPos) {
            const Real v = KT::val(kmax);
            const bool better = !found || v > best || (v == best && lmin < best_lex);
            found = true;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                const Real xt = __shfl_sync(kFull, xc[t], who);
                W.x[t] = better ? xt : W.x[t];
            }
            const unsigned bm = __shfl_sync(kFull, mask, who);
            const int bs = __shfl_sync(kFull, sg, who);
            best_mask = better ? bm : best_mask;
            best_sg = better ? bs : best_sg;
            best_lex = better ? lmin : best_lex;
            best = better ? v : best;
        }
    }
    if (!found) return false;
    if (W.lane == 0) {
        unsigned mk = best_mask;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int a = __ffs(mk) - 1;
            mk &= mk - 1u;
            W.defs[D - K + r] = 2 * a + ((best_sg >> r) & 1);
        }
    }
    return true;
}

// The level-(K-1) frame: the hyperplane of slot f inside the level-K subspace (the
// whole space, p = 0 and E = I, when K == D).  False if g's normal is orthogonal to
// the subspace (then the violated g excludes all of it).
template <typename Real, int D, int K, typename WT>
__device__ __forceinline__ bool child_frame(WT& W, int f) {
    constexpr int S = WT::kS;
    const Real* F = W.fr + frame_off<D>(K < D ? K : 1);
    Real g[D];
#pragma unroll
    for (int t = 0; t < D; ++t) g[t] = W.s[t * S + f];
    Real r = W.s[D * S + f];
    Real A[K];
    if constexpr (K == D) {
#pragma unroll
        for (int i = 0; i < K; ++i) A[i] = g[i];
    } else {
#pragma unroll
        for (int t = 0; t < D; ++t) r -= g[t] * F[t];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            Real v = Real(0);
#pragma unroll
            for (int t = 0; t < D; ++t) v += g[t] * F[D * (1 + i) + t];
            A[i] = v;
        }
    }
    int J = 0;
    Real aJ = real_abs(A[0]), AJ = A[0];
#pragma unroll
    for (int i = 1; i < K; ++i) {
        const bool take = real_abs(A[i]) > aJ;
        J = take ? i : J;
        aJ = take ? real_abs(A[i]) : aJ;
        AJ = take ? A[i] : AJ;
    }
    if (!(aJ > Real(0))) return false;
    const Real inv = real_rcp(AJ);
    __syncwarp();  // every lane is done with the previous frame of this level
    if (W.lane < D) {
        const int t = W.lane;
        Real* C = W.fr + frame_off<D>(K - 1);
        Real EJt, pt;
        if constexpr (K == D) {
            EJt = (t == J) ? Real(1) : Real(0);
            pt = Real(0);
        } else {
            EJt = F[D * (1 + J) + t];
            pt = F[t];
        }
        C[t] = pt + (r * inv) * EJt;
        int n = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            if (i == J) continue;
            Real Eit;
            if constexpr (K == D) Eit = (t == i) ? Real(1) : Real(0);
            else Eit = F[D * (1 + i) + t];
            C[D * (1 + n) + t] = Eit - (A[i] * inv) * EJt;
            ++n;
        }
    }
    __syncwarp();
    return true;
}

// The LP on the level-K subspace over the stage slots 0..limit-1 (the box and the
// constraints visited before slot limit).  Level D starts from the current x (the
// box corner); lower levels find their own start.  False if infeasible.
template <typename Real, int D, int K, typename WT>
__device__ __forceinline__ bool solve_level(WT& W, int limit) {
    constexpr int S = WT::kS;
    if constexpr (K == 1) {
        // Eqs. 3, 4 on the line p + t e, e oriented so that the objective's end is the
        // right end (the left end of E_0 when c is perpendicular to the line)
        const Real* F = W.fr + frame_off<D>(1);
        Real p[D], e[D], ce = Real(0);
#pragma unroll
        for (int t = 0; t < D; ++t) {
            p[t] = F[t];
            e[t] = F[D + t];
            ce += W.c[t] * e[t];
        }
        const Real sgn = ce > Real(0) ? Real(1) : Real(-1);
#pragma unroll
        for (int t = 0; t < D; ++t) e[t] *= sgn;
        Real thi = real_inf<Real>(), tlo = -real_inf<Real>();
        const Real ninf = -real_inf<Real>();
        int phi = kNoPos;
        for (int f = W.lane; f < limit; f += 32) {
            Real num = W.s[D * S + f], den = Real(0);
#pragma unroll
            for (int t = 0; t < D; ++t) {
                const Real gt = W.s[t * S + f];
                num -= gt * p[t];
                den += gt * e[t];
            }
            den = den + Real(0);  // -0 counts as +0: a parallel constraint is a right bound
            const Real tau = real_div<Real>(num, den);
            const bool right = den >= Real(0);
            const bool take = right && (tau < thi);
            thi = take ? tau : thi;
            phi = take ? f : phi;
            tlo = real_max<Real>(tlo, right ? ninf : tau);
        }
        warp_reduce_1dlp<Real>(thi, phi, tlo);
        if (!(tlo <= thi)) return false;  // empty interval, or a parallel constraint excludes the line
#pragma unroll
        for (int t = 0; t < D; ++t) W.x[t] = p[t] + thi * e[t];
        if (W.lane == 0) W.defs[D - 1] = phi;
        return true;
    } else {
        if constexpr (K < D) {
            if (!box_start<Real, D, K>(W)) return false;
        }
        int k = 2 * D;
        while (k < limit) {
            const int q = k + W.lane;
            const bool v = q < limit && violates_n<Real, D, S>(W.s, q, W.x, W.eps);
            const unsigned bal = __ballot_sync(kFull, v);
            if (bal == 0u) {
                k += 32;
                continue;
            }
            const int f = k + __ffs(bal) - 1;
            k = f + 1;
            if constexpr (K == D) ++W.nviol;
            if (!child_frame<Real, D, K>(W, f)) return false;
            if (!solve_level<Real, D, K - 1>(W, f)) return false;
            if (W.lane == 0) W.defs[D - K] = f;
        }
        return true;
    }
}

template <int D, int S = kStageN>
__device__ __forceinline__ void write_box_n(const ParamsN& P, float* s, int lane) {
    if (lane < 2 * D) {
        const int axis = lane >> 1;
        const float sg = (lane & 1) ? -1.0f : 1.0f;
        float bv = 0.0f;
#pragma unroll
        for (int t = 0; t < D; ++t) {
            s[t * S + lane] = (t == axis) ? sg : 0.0f;
            if (t == axis) bv = (lane & 1) ? -P.box[2 * t] : P.box[2 * t + 1];
        }
        s[D * S + lane] = bv;
    }
}

// Warp staging of an LP with m <= 1024 - 2D constraints (key domain <= 1024 bits, one
// bitmap word per lane): slot 2D + rank of the constraint's key.
template <int D>
__device__ __forceinline__ void stage_lp_n(const ParamsN& P, const VisitOrder& vo, int m, long long base, float* s,
                                           unsigned* bm, int lane) {
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
            const int slot = 2 * D + pe + __popc(we & ((1u << (e & 31u)) - 1u));
#pragma unroll
            for (int t = 0; t < D; ++t) cp_async4(const_cast<float*>(s) + t * kStageN + slot, P.a[t] + base + q);
            cp_async4(s + D * kStageN + slot, P.b + base + q);
        }
    }
}

// Constraint id of a stage slot for out_def: -1 - plane for the box, otherwise the
// index of the constraint staged there.
template <int D>
__device__ __forceinline__ int slot_id_n(int slot, const VisitOrder& vo, const unsigned* bm, int lane) {
    if (slot < 2 * D) return -1 - slot;
    const uint64_t dw = vo.domain() >> 5;
    const int nwords = dw > 0 ? static_cast<int>(dw) : 1;
    return static_cast<int>(vo.dec(bitmap_select(bm, nwords, slot - 2 * D, lane)));
}

template <typename Real, int D>
__device__ __forceinline__ void write_bad_n(const ParamsN& P, int64_t lp, unsigned bits) {
    atomicOr(P.ws + kWsError, static_cast<unsigned long long>(bits));
    P.out_status[lp] = kBadInput;
    Real* out = reinterpret_cast<Real*>(P.out_x);
    const Real nan = real_inf<Real>() - real_inf<Real>();
#pragma unroll
    for (int t = 0; t < D; ++t) out[D * lp + t] = nan;
    if (P.out_nviol) P.out_nviol[lp] = 0;
    if (P.out_def)
#pragma unroll
        for (int t = 0; t < D; ++t) P.out_def[D * lp + t] = INT32_MIN;
}

// Seidel's method on one staged LP by one warp; writes the LP's outputs.
template <typename Real, int D, int S = kStageN>
__device__ void drive_lp_n(const ParamsN& P, int64_t lp, int m, const VisitOrder& vo, const float* s, Real* fr,
                           int* defs, const unsigned* bm, int lane) {
    WarpN<Real, D, S> W;
    W.s = s;
    W.fr = fr;
    W.defs = defs;
    W.lane = lane;
    W.nviol = 0;
    W.eps = (sizeof(Real) == 4) ? Real(P.eps32) : Real(P.eps64);
    bool bad = false;
#pragma unroll
    for (int t = 0; t < D; ++t) {
        const float ct = __ldg(P.obj + D * lp + t);
        bad |= !(fabsf(ct) <= 3.402823466e38f);
        W.c[t] = ct;
        W.x[t] = ct >= 0.0f ? Real(P.box[2 * t + 1]) : Real(P.box[2 * t]);
        if (lane == t) defs[t] = 2 * t + (ct >= 0.0f ? 0 : 1);  // the box corner that maximises c
    }
    if (P.check_finite) {
        bool nf = false;
        for (int i = lane; i < m; i += 32)
#pragma unroll
            for (int t = 0; t <= D; ++t) nf |= !(fabsf(s[t * S + 2 * D + i]) <= 3.402823466e38f);
        bad |= __any_sync(kFull, nf);
    }
    __syncwarp();
    int status = -1;
    if (bad) status = kBadInput;
    else if (!solve_level<Real, D, D>(W, 2 * D + m)) status = kInfeasible;
    __syncwarp();
    const bool none = status == kInfeasible || status == kBadInput;
    int ids[D];
#pragma unroll
    for (int t = 0; t < D; ++t) ids[t] = INT32_MIN;
    if (P.out_def && !none) {
#pragma unroll
        for (int t = 0; t < D; ++t) ids[t] = slot_id_n<D>(defs[t], vo, bm, lane);
    }
    if (lane == 0) {
        if (status < 0) {
            bool box_def = false;
#pragma unroll
            for (int t = 0; t < D; ++t) box_def |= defs[t] < 2 * D;
            status = box_def ? kBoxBounded : kOptimal;
        }
        Real* out = reinterpret_cast<Real*>(P.out_x);
        const Real nan = real_inf<Real>() - real_inf<Real>();
#pragma unroll
        for (int t = 0; t < D; ++t) out[D * lp + t] = none ? nan : W.x[t];
        P.out_status[lp] = status;
        if (P.out_nviol) P.out_nviol[lp] = W.nviol;
        if (P.out_def)
#pragma unroll
            for (int t = 0; t < D; ++t) P.out_def[D * lp + t] = ids[t];
    }
}

// One warp's loop over a queue: grab spans of LP indices (doubling after a grab
// without LPs of the class, halving after one with more than the target), stage and
// solve the LPs of size (lo, hi] among them.
template <typename Real, int D, int S = kStageN, bool kLarge = false>
__device__ void warp_queue_n(const ParamsN& P, unsigned long long* head, long long lo, long long hi, float* s,
                             Real* fr, int* defs, unsigned* bm, int lane, int* pre = nullptr) {
    constexpr int kCap = (kLarge ? S : kHalfN) - 2 * D;
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
        unsigned todo = __ballot_sync(kFull, in && mm_l > lo && mm_l <= hi);
        const int found = __popc(todo);
        span = found == 0 ? min(2 * span, 32) : (found > P.chunk ? max(span >> 1, 1) : span);
        while (todo != 0u) {
            const int i = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int64_t lp = start + i;
            const long long base = __shfl_sync(kFull, off_l, i);
            const long long mm = __shfl_sync(kFull, mm_l, i);
            if (mm < 0 || mm > kCap) {
                if (lane == 0) write_bad_n<Real, D>(P, lp, mm < 0 ? kDevErrBadOffsets : kDevErrTooLargeN);
                continue;
            }
            const int m = static_cast<int>(mm);
            VisitOrder vo;
            warp_visit_order(vo, P.seed + static_cast<uint64_t>(lp), static_cast<uint32_t>(m), lane);
            write_box_n<D, S>(P, s, lane);
            if constexpr (kLarge) {
                stage_ranks_warp(vo, m, bm, pre, lane, [&](int r, int q) {
                    const int slot = 2 * D + r;
#pragma unroll
                    for (int t = 0; t < D; ++t) cp_async4(s + t * S + slot, P.a[t] + base + q);
                    cp_async4(s + D * S + slot, P.b + base + q);
                });
            } else {
                stage_lp_n<D>(P, vo, m, base, s, bm, lane);
            }
            cp_async_wait_all();
            __syncwarp();
            drive_lp_n<Real, D, S>(P, lp, m, vo, s, fr, defs, bm, lane);
            __syncwarp();  // all lanes are done with the stage before it is overwritten
        }
    }
}

template <typename Real, int D>
__global__ void __launch_bounds__(kWarpsN * 32, (min_ctas_n<D, Real>())) seidel_nd_kernel(const ParamsN P) {
    extern __shared__ __align__(16) unsigned char smem_n[];
    float* stage = reinterpret_cast<float*>(smem_n);
    Real* frames = reinterpret_cast<Real*>(smem_n + sizeof(float) * (D + 1) * kStageN);
    int* defs = reinterpret_cast<int*>(frames + kWarpsN * kFrameReals<D>);
    unsigned* bms = reinterpret_cast<unsigned*>(defs + kWarpsN * D);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned long long* ws = P.ws;
    Real* fr = frames + warp * kFrameReals<D>;
    int* df = defs + warp * D;
    unsigned* bm = bms + warp * 32;
    // mid-size LPs: warps 0 and 1, half a stage each
    if (warp < 2)
        warp_queue_n<Real, D>(P, ws + kWsHeadMid, kQuarterN - 2 * D, kHalfN - 2 * D, stage + warp * kHalfN, fr, df,
                              bm, lane);
    __syncthreads();
    // small LPs (and negative sizes): every warp, a quarter of the stage each
    warp_queue_n<Real, D>(P, ws + kWsHeadSmall, -(1ll << 62), kQuarterN - 2 * D, stage + warp * kQuarterN, fr, df,
                          bm, lane);
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

// The large-LP kernel: one warp per CTA, a stage of kStageNL slots per array and a key
// bitmap for domains up to 4^7 = 16384 bits, in dynamic shared memory.
constexpr int kStageNL = 8192;
constexpr int kWordsNL = 512;
constexpr int kWsDoneLargeN = 5;  // workspace word: large-LP CTAs that have finished

template <int D, typename Real> constexpr size_t smem_bytes_nl() {
    return sizeof(float) * (D + 1) * kStageNL + sizeof(Real) * kFrameReals<D> + sizeof(int) * D +
           sizeof(unsigned) * kWordsNL + sizeof(int) * kWordsNL;
}

// LPs above the half stage: one warp per CTA; LPs above kStageNL - 2d constraints are
// reported as too large.  Runs after seidel_nd_kernel on the same stream, with its own
// queue head and done counter.
template <typename Real, int D>
__global__ void __launch_bounds__(32, 1) seidel_nd_large_kernel(const ParamsN P) {
    extern __shared__ __align__(16) unsigned char smem_nl[];
    float* stage = reinterpret_cast<float*>(smem_nl);
    Real* fr = reinterpret_cast<Real*>(smem_nl + sizeof(float) * (D + 1) * kStageNL);
    int* df = reinterpret_cast<int*>(fr + kFrameReals<D>);
    unsigned* bm = reinterpret_cast<unsigned*>(df + D);
    int* pre = reinterpret_cast<int*>(bm + kWordsNL);
    const int lane = threadIdx.x;
    unsigned long long* ws = P.ws;
    warp_queue_n<Real, D, kStageNL, true>(P, ws + kWsHeadBig, kHalfN - 2 * D, 1ll << 62, stage, fr, df, bm, lane,
                                          pre);
    if (lane == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(ws + kWsDoneLargeN, 1ull);
        if (prev == static_cast<unsigned long long>(gridDim.x) - 1ull) {
            atomicExch(ws + kWsHeadBig, 0ull);
            atomicExch(ws + kWsDoneLargeN, 0ull);
        }
    }
}

}  // namespace lp2d

namespace {

using lp2d::report_error;

bool aligned_n(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Opt in to more than 48 KB of dynamic shared memory once per kernel and device.
template <typename Real, int D>
int launch_nd(const lp2d::ParamsN& p, int ctas_per_sm_cap, int64_t n_lp, cudaStream_t s) {
    constexpr size_t bytes = lp2d::smem_bytes_n<D, Real>();
    auto kernel = lp2d::seidel_nd_kernel<Real, D>;
    static std::mutex mu;
    static bool ready[64] = {};
    static bool ready_large[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_error(LP2D_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return report_error(LP2D_ERR_CUDA, "device ordinal %d out of range", dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready[dev]) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
            if (e != cudaSuccess) return report_error(LP2D_ERR_CUDA, "shared memory opt-in: %s", cudaGetErrorString(e));
            ready[dev] = true;
        }
    }
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, lp2d::kWarpsN * 32, bytes);
    if (e != cudaSuccess) return report_error(LP2D_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    if (per_sm < 1) return report_error(LP2D_ERR_CUDA, "d-dimensional kernel cannot be resident");
    if (ctas_per_sm_cap > 0 && ctas_per_sm_cap < per_sm) per_sm = ctas_per_sm_cap;
    long long grid = static_cast<long long>(sms) * per_sm;
    const long long useful = (n_lp + lp2d::kWarpsN - 1) / lp2d::kWarpsN;
    if (grid > useful) grid = useful;
    if (grid < 1) grid = 1;
    kernel<<<static_cast<int>(grid), lp2d::kWarpsN * 32, bytes, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(LP2D_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    // LPs above the half stage: one CTA per SM, each a warp with a large stage
    constexpr size_t lbytes = lp2d::smem_bytes_nl<D, Real>();
    auto large = lp2d::seidel_nd_large_kernel<Real, D>;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready_large[dev]) {
            e = cudaFuncSetAttribute(large, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(lbytes));
            if (e != cudaSuccess)
                return report_error(LP2D_ERR_CUDA, "large-LP shared memory opt-in: %s", cudaGetErrorString(e));
            ready_large[dev] = true;
        }
    }
    large<<<static_cast<int>(std::min<long long>(sms, n_lp)), 32, lbytes, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(LP2D_ERR_CUDA, "large-LP kernel launch: %s", cudaGetErrorString(e));
    return LP2D_OK;
}

template <typename Real>
int launch_nd_dim(int d, const lp2d::ParamsN& p, int cap, int64_t n_lp, cudaStream_t s) {
    switch (d) {
        case 2: return launch_nd<Real, 2>(p, cap, n_lp, s);
        case 3: return launch_nd<Real, 3>(p, cap, n_lp, s);
        case 4: return launch_nd<Real, 4>(p, cap, n_lp, s);
        default: return launch_nd<Real, 5>(p, cap, n_lp, s);
    }
}

}  // namespace

extern "C" int lpnd_solve_batch(int d, const float* const* a, const float* b, const int64_t* offsets, int64_t n_lp,
                                const float* obj, const float* box, void* out_x, int32_t* out_status,
                                const lp2d_options* opt_in, void* workspace, size_t workspace_bytes,
                                lp2d_stream_t stream) {
    lp2d_options opt;
    if (opt_in) opt = *opt_in;
    else lp2d_default_options(&opt);
    if (d < 2 || d > LPND_MAX_DIM) return report_error(LP2D_ERR_INVALID_ARGUMENT, "d = %d is outside 2..%d", d,
                                                       LPND_MAX_DIM);
    if (n_lp < 0) return report_error(LP2D_ERR_INVALID_ARGUMENT, "n_lp = %lld < 0", (long long)n_lp);
    if (opt.precision != LP2D_PREC_FP32 && opt.precision != LP2D_PREC_FP64)
        return report_error(LP2D_ERR_UNSUPPORTED, "the d-dimensional solver runs in FP32 or FP64");
    if (opt.schedule != LP2D_SCHED_PERSISTENT)
        return report_error(LP2D_ERR_UNSUPPORTED, "the d-dimensional solver has the persistent schedule only");
    if (opt.chunk_small < 0 || !(opt.eps >= 0.0f) || !std::isfinite(opt.eps))
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "bad tuning parameter or eps");
    if (!box) return report_error(LP2D_ERR_INVALID_ARGUMENT, "box is NULL");
    for (int t = 0; t < d; ++t) {
        if (!std::isfinite(box[2 * t]) || !std::isfinite(box[2 * t + 1]))
            return report_error(LP2D_ERR_INVALID_ARGUMENT, "box must be finite");
        if (!(box[2 * t] < box[2 * t + 1]))
            return report_error(LP2D_ERR_INVALID_ARGUMENT, "box needs min < max on every axis (axis %d)", t);
    }
    if (n_lp == 0) return LP2D_OK;
    if (!a || !b || !offsets || !obj || !out_x || !out_status)
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "NULL data pointer");
    for (int t = 0; t < d; ++t)
        if (!a[t] || !aligned_n(a[t], 4))
            return report_error(LP2D_ERR_INVALID_ARGUMENT, "a[%d] is NULL or misaligned", t);
    const size_t out_align = (opt.precision == LP2D_PREC_FP64) ? 8 : 4;
    if (!aligned_n(b, 4) || !aligned_n(obj, 4) || !aligned_n(offsets, 8) || !aligned_n(out_x, out_align) ||
        !aligned_n(out_status, 4) || (opt.out_nviol && !aligned_n(opt.out_nviol, 4)) ||
        (opt.out_def && !aligned_n(opt.out_def, 4)))
        return report_error(LP2D_ERR_INVALID_ARGUMENT, "misaligned pointer");
    const size_t need = sizeof(unsigned long long) * lp2d::kWsWords;
    if (!workspace) return report_error(LP2D_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", need);
    if (workspace_bytes < need || !aligned_n(workspace, 8))
        return report_error(LP2D_ERR_WORKSPACE, "workspace needs %zu bytes, 8-byte aligned", need);

    lp2d::ParamsN p{};
    for (int t = 0; t < d; ++t) p.a[t] = a[t];
    p.b = b;
    p.offsets = offsets;
    p.n_lp = n_lp;
    p.obj = obj;
    for (int t = 0; t < 2 * d; ++t) p.box[t] = box[t];
    p.seed = opt.seed;
    p.out_x = out_x;
    p.out_status = out_status;
    p.out_nviol = opt.out_nviol;
    p.out_def = opt.out_def;
    p.ws = reinterpret_cast<unsigned long long*>(workspace);
    p.eps32 = opt.eps > 0.0f ? opt.eps : 1e-6f;
    p.eps64 = opt.eps > 0.0f ? static_cast<double>(opt.eps) : 1e-12;
    p.chunk = opt.chunk_small > 0
                  ? (opt.chunk_small < lp2d::kMaxChunkSmall ? opt.chunk_small : lp2d::kMaxChunkSmall)
                  : lp2d::kDefaultChunkSmall;
    p.check_finite = opt.check_finite ? 1 : 0;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (opt.precision == LP2D_PREC_FP64) return launch_nd_dim<double>(d, p, opt.ctas_per_sm, n_lp, s);
    return launch_nd_dim<float>(d, p, opt.ctas_per_sm, n_lp, s);
}
