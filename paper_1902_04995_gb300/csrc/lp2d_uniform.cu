// lp2d_uniform.cu -- the plain uniform-launch solver and the visit-order kernel.
//
// One thread per LP, every thread stepping through its own constraints in visit
// order and reading them from global memory: the mapping of the paper's naive
// kernel (Sec. 3: "each LP is assigned to a core/thread"), kept as the comparator
// of the persistent solver.  In FP64 it is the reference-precision GPU path.
// The 1-D LP of a violation at position k re-derives pi(j) for every j < k rather
// than keeping a per-thread copy of the order.
#include "lp2d_internal.h"

namespace lp2d {

template <typename Real>
__global__ void __launch_bounds__(128) seidel_uniform_kernel(const Params P) {
    const int64_t lp = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (lp >= P.n_lp) return;
    Real* out = reinterpret_cast<Real*>(P.out_xy);
    const Real nan = real_inf<Real>() - real_inf<Real>();
    const int64_t base = __ldg(P.offsets + lp);
    const int64_t m64 = __ldg(P.offsets + lp + 1) - base;
    if (m64 < 0 || m64 > 0x7fffffffll) {
        if (P.ws) atomicOr(P.ws + kWsError, static_cast<unsigned long long>(kDevErrBadOffsets));
        P.out_status[lp] = kBadInput;
        out[2 * lp] = out[2 * lp + 1] = nan;
        return;
    }
    const int m = static_cast<int>(m64);
    const float* __restrict__ gax = P.ax + base;
    const float* __restrict__ gay = P.ay + base;
    const float* __restrict__ gbb = P.b + base;
    const float cxf = __ldg(P.obj + 2 * lp), cyf = __ldg(P.obj + 2 * lp + 1);
    bool bad = !(fabsf(cxf) <= 3.402823466e38f) || !(fabsf(cyf) <= 3.402823466e38f);
    if (P.check_finite) {
        float fin = 0.0f;
        for (int q = 0; q < m; ++q) {
            fin = fmaf(__ldg(gax + q), 0.0f, fin);
            fin = fmaf(__ldg(gay + q), 0.0f, fin);
            fin = fmaf(__ldg(gbb + q), 0.0f, fin);
        }
        bad = bad || (fin != fin);
    }
    if (bad) {
        P.out_status[lp] = kBadInput;
        out[2 * lp] = out[2 * lp + 1] = nan;
        return;
    }
    VisitOrder vo;
    vo.init(P.seed + static_cast<uint64_t>(lp), static_cast<uint32_t>(m));
    bool werr = false;
    const Real cx = cxf, cy = cyf;
    const Real eps = (sizeof(Real) == 4) ? Real(P.eps32) : Real(P.eps64);

    Real vx = (cx >= Real(0)) ? Real(P.xmax) : Real(P.xmin);
    Real vy = (cy >= Real(0)) ? Real(P.ymax) : Real(P.ymin);
    int d0 = (cx >= Real(0)) ? -4 : -3;
    int d1 = (cy >= Real(0)) ? -2 : -1;
    int status = -1;
    int nviol = 0;

    for (int k = 0; k < m; ++k) {
        const uint32_t h = vo.fwd(static_cast<uint32_t>(k), werr);
        const Real hx = __ldg(gax + h), hy = __ldg(gay + h), hb = __ldg(gbb + h);
        const Real s = hx * vx + hy * vy - hb;
        const Real tol = eps * (real_abs(hx * vx) + real_abs(hy * vy) + real_abs(hb));
        if (!(s > tol)) continue;
        const Real nrm2 = hx * hx + hy * hy;
        if (nrm2 == Real(0)) {
            status = kInfeasible;
            d0 = k;
            break;
        }
        const Real sc0 = hb / nrm2;
        const Real p0x = hx * sc0, p0y = hy * sc0;
        const Real ux = -hy, uy = hx;
        Real thi = real_inf<Real>(), tlo = -real_inf<Real>();
        int phi = kNoPos, plo = kNoPos;
        bool par = false;
        // earlier constraints in visit-position order: box sides (-4..-1), then 0..k-1
        for (int j = -4; j < k && !par; ++j) {
            Real gx, gy, gb;
            if (j < 0) {
                box_side<Real>(P, j + 4, gx, gy, gb);
            } else {
                const uint32_t g = vo.fwd(static_cast<uint32_t>(j), werr);
                gx = __ldg(gax + g);
                gy = __ldg(gay + g);
                gb = __ldg(gbb + g);
            }
            const Real den = gx * ux + gy * uy;
            const Real num = gb - (gx * p0x + gy * p0y);
            if (den > Real(0)) {
                const Real t = real_div<Real>(num, den);
                if (t < thi) { thi = t; phi = j; }
            } else if (den < Real(0)) {
                const Real t = real_div<Real>(num, den);
                if (t > tlo) { tlo = t; plo = j; }
            } else if (num < Real(0)) {
                par = true;
            }
        }
        ++nviol;
        if (par || tlo > thi) {
            status = kInfeasible;
            d0 = k;
            break;
        }
        const Real cu = cx * ux + cy * uy;
        const bool right = cu > Real(0);
        const Real t = right ? thi : tlo;
        vx = p0x + t * ux;
        vy = p0y + t * uy;
        d0 = k;
        d1 = right ? phi : plo;
    }
    if (werr && P.ws) atomicOr(P.ws + kWsError, static_cast<unsigned long long>(kDevErrWalkLimit));
    if (status < 0) status = (d0 < 0 || d1 < 0) ? kBoxBounded : kOptimal;
    if (status == kInfeasible) {
        out[2 * lp] = out[2 * lp + 1] = nan;
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

__global__ void visit_order_kernel(uint64_t seed, int64_t m, int64_t* out) {
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= m) return;
    VisitOrder vo;
    vo.init(seed, static_cast<uint32_t>(m));
    bool werr = false;
    const uint32_t q = vo.fwd(static_cast<uint32_t>(k), werr);
    out[k] = werr ? -1 : static_cast<int64_t>(q);
}

static int uniform_grid(int64_t n_lp) { return static_cast<int>((n_lp + 127) / 128); }

cudaError_t launch_uniform_f32(const Params& p, cudaStream_t s) {
    seidel_uniform_kernel<float><<<uniform_grid(p.n_lp), 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_uniform_f64(const Params& p, cudaStream_t s) {
    seidel_uniform_kernel<double><<<uniform_grid(p.n_lp), 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_visit_order(uint64_t seed, int64_t m, int64_t* out, cudaStream_t s) {
    const int64_t blocks = (m + 255) / 256;
    visit_order_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(seed, m, out);
    return cudaGetLastError();
}

}  // namespace lp2d
