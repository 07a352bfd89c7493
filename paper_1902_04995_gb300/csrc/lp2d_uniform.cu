// lp2d_uniform.cu -- the plain uniform-launch solver and the visit-order kernel.
//
// One thread per LP, every thread stepping through its own constraints in visit
// order and reading them from global memory: the mapping of the paper's naive
// kernel (Sec. 3 assigns each LP to one thread), kept as the comparator of the
// persistent solver.  In FP64 it is the reference-precision GPU path.
// The visit order is the increasing order of the constraints' Feistel keys, so the
// thread scans the key domain upward and skips keys whose constraint index is >= m;
// the 1-D LP of a violation at key e rescans the keys below e.
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
    if (m64 < 0 || m64 > (1ll << 30)) {
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
    const uint32_t dom = static_cast<uint32_t>(vo.domain());  // <= 2^30
    const Real cx = cxf, cy = cyf;
    const Real eps = (sizeof(Real) == 4) ? Real(P.eps32) : Real(P.eps64);

    Real vx = (cx >= Real(0)) ? Real(P.xmax) : Real(P.xmin);
    Real vy = (cy >= Real(0)) ? Real(P.ymax) : Real(P.ymin);
    int d0 = (cx >= Real(0)) ? 0 : 1;  // tags of the defining pair: box sides 0..3, else 4 + key
    int d1 = (cy >= Real(0)) ? 2 : 3;
    int status = -1;
    int nviol = 0;

    for (uint32_t e = 0; e < dom; ++e) {
        const uint32_t h = vo.dec(e);
        if (h >= static_cast<uint32_t>(m)) continue;
        const Real hx = __ldg(gax + h), hy = __ldg(gay + h), hb = __ldg(gbb + h);
        const Real s = hx * vx + hy * vy - hb;
        const Real tol = eps * (real_abs(hx * vx) + real_abs(hy * vy) + real_abs(hb));
        if (!(s > tol)) continue;
        const Real nrm2 = hx * hx + hy * hy;
        if (nrm2 == Real(0)) {
            status = kInfeasible;
            break;
        }
        const Real sc0 = hb / nrm2;
        const Real p0x = hx * sc0, p0y = hy * sc0;
        const Real ux = -hy, uy = hx;
        Real thi = real_inf<Real>(), tlo = -real_inf<Real>();
        int phi = kNoPos, plo = kNoPos;
        bool par = false;
        // earlier constraints in visit order: box sides (tags 0..3), then keys below e
        for (int j = -4; j < static_cast<int>(e) && !par; ++j) {
            Real gx, gy, gb;
            if (j < 0) {
                box_side<Real>(P, j + 4, gx, gy, gb);
            } else {
                const uint32_t g = vo.dec(static_cast<uint32_t>(j));
                if (g >= static_cast<uint32_t>(m)) continue;
                gx = __ldg(gax + g);
                gy = __ldg(gay + g);
                gb = __ldg(gbb + g);
            }
            const Real den = gx * ux + gy * uy;
            const Real num = gb - (gx * p0x + gy * p0y);
            if (den > Real(0)) {
                const Real t = real_div<Real>(num, den);
                if (t < thi) { thi = t; phi = j + 4; }
            } else if (den < Real(0)) {
                const Real t = real_div<Real>(num, den);
                if (t > tlo) { tlo = t; plo = j + 4; }
            } else if (num < Real(0)) {
                par = true;
            }
        }
        ++nviol;
        if (par || tlo > thi) {
            status = kInfeasible;
            break;
        }
        const Real cu = cx * ux + cy * uy;
        const bool right = cu > Real(0);
        const Real t = right ? thi : tlo;
        vx = p0x + t * ux;
        vy = p0y + t * uy;
        d0 = 4 + static_cast<int>(e);
        d1 = right ? phi : plo;
    }
    if (status < 0) status = (d0 < 4 || d1 < 4) ? kBoxBounded : kOptimal;
    if (status == kInfeasible) {
        out[2 * lp] = out[2 * lp + 1] = nan;
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

// pi of one LP: scan the key domain upward in blocks of 1024 keys; the valid keys of
// a block (constraint index < m) take the next positions in order.  One CTA.
__global__ void __launch_bounds__(1024) visit_order_kernel(uint64_t seed, int64_t m, int64_t* out) {
    __shared__ int s_cnt[32];
    VisitOrder vo;
    vo.init(seed, static_cast<uint32_t>(m));
    const uint64_t dom = vo.domain();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t base = 0;
    for (uint64_t e0 = 0; e0 < dom; e0 += 1024) {
        const uint64_t e = e0 + static_cast<uint64_t>(tid);
        uint32_t q = 0;
        bool valid = false;
        if (e < dom) {
            q = vo.dec(static_cast<uint32_t>(e));
            valid = q < static_cast<uint32_t>(m);
        }
        const unsigned bal = __ballot_sync(kFull, valid);
        if (lane == 0) s_cnt[warp] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < 32; ++w) {
            before += (w < warp) ? s_cnt[w] : 0;
            total += s_cnt[w];
        }
        if (valid) out[base + before + __popc(bal & ((1u << lane) - 1u))] = static_cast<int64_t>(q);
        base += total;
        __syncthreads();
    }
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
    visit_order_kernel<<<1, 1024, 0, s>>>(seed, m, out);
    return cudaGetLastError();
}

}  // namespace lp2d
