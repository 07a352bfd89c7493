// lp2d_device.cuh -- device building blocks of the batched 2-D Seidel solver (sm_103a).
//
// Seidel's randomized incremental LP (Sec. 2.1 of Charlton, Maddock & Richmond,
// arXiv 1902.04995): visit the constraints of an LP in random order; keep the
// optimum while it satisfies the visited constraint; otherwise move it onto that
// constraint's line with a 1-D LP over all earlier constraints (Eq. 3: the largest
// left bound, Eq. 4: the smallest right bound; empty interval = infeasible).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lp2d {

constexpr int kOptimal = 0;
constexpr int kInfeasible = 1;
constexpr int kBoxBounded = 2;
constexpr int kBadInput = 3;
constexpr int kNoPos = 0x7fffffff;
constexpr unsigned kFull = 0xffffffffu;

// Bits of the device error word (same values as LP2D_DEVERR_* in lp2d.h).
constexpr unsigned kDevErrBadOffsets = 1u;

// Workspace words of the persistent schedule.
constexpr int kWsHeadBig = 0;    // next LP index for CTA teams
constexpr int kWsHeadSmall = 1;  // next LP index for single warps
constexpr int kWsDone = 2;       // CTAs that have finished
constexpr int kWsError = 3;      // device error word
constexpr int kWsHeadMid = 4;    // next LP index for warps with half a CTA stage
constexpr int kWsHeadTiny = 6;   // next LP index for single lanes
constexpr int kWsWords = 32;     // 256 bytes

struct Params {
    const float* __restrict__ ax;
    const float* __restrict__ ay;
    const float* __restrict__ b;
    const int64_t* __restrict__ offsets;
    int64_t n_lp;
    const float* __restrict__ obj;
    float xmin, xmax, ymin, ymax;
    uint64_t seed;
    void* out_xy;
    int32_t* out_status;
    int32_t* out_nviol;
    int32_t* out_def;
    unsigned long long* ws;  // persistent-schedule workspace (kWsWords words)
    float eps32;
    double eps64;
    float tau;
    int chunk_big;
    int chunk_small;
    int check_finite;
    int team_min;   // 1-D LPs over at least this many stage slots get the CTA's helper warps
    int prefetch;   // non-zero: bulk-prefetch each grabbed LP's constraints into L2
    int lane_max_m;  // FP32: LPs of at most this many constraints go to single lanes (0: none)
};

// ------------------------------------------------------------------ visit order
// A random visit order gives Seidel's method its expected O(m) time (Sec. 2.1).
// LP l visits its constraints in increasing order of a key E(q): E is a 4-round
// balanced Feistel network on 2h bits (2h >= ceil(log2 m), h >= 1), a bijection of
// [0, 4^h), so keys are distinct.  Round key r is the low word of output r+1 of
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) seeded with seed + l; the round
// function is the top h bits of (R xor K) * 0x9E3779B1 (mod 2^32).
// Positions follow from keys without any loop: the visit position of q is the
// number of constraints with a smaller key (a rank in a bitmap of the keys), and
// scanning the key domain upward, skipping keys whose constraint index is >= m,
// lists the constraints in visit order.
__device__ __forceinline__ uint64_t splitmix64_output(uint64_t seed, uint32_t r) {
    uint64_t z = seed + static_cast<uint64_t>(r + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct VisitOrder {
    uint32_t k0, k1, k2, k3;
    uint32_t h;      // bits per half
    uint32_t mask;   // (1 << h) - 1
    uint32_t m;      // number of constraints
    uint32_t up;     // 2^h
    uint32_t down;   // 2^(32-h)

    __device__ __forceinline__ void init_shape(uint32_t m_) {
        m = m_;
        const uint32_t bits = (m_ <= 1u) ? 0u : 32u - static_cast<uint32_t>(__clz(static_cast<int>(m_ - 1u)));
        h = (bits + 1u) >> 1;
        if (h < 1u) h = 1u;
        mask = (1u << h) - 1u;  // h <= 16 since m < 2^31
        up = 1u << h;
        down = 1u << (32u - h);
    }

    __device__ __forceinline__ void init(uint64_t seed, uint32_t m_) {
        init_shape(m_);
        k0 = static_cast<uint32_t>(splitmix64_output(seed, 0));
        k1 = static_cast<uint32_t>(splitmix64_output(seed, 1));
        k2 = static_cast<uint32_t>(splitmix64_output(seed, 2));
        k3 = static_cast<uint32_t>(splitmix64_output(seed, 3));
    }

    // Size of the key domain, 4^h.
    __device__ __forceinline__ uint64_t domain() const { return 1ull << (2u * h); }

    // Round function: the top h bits of the 32-bit product, taken as the high word of
    // a second multiply by 2^h; the shifts of this struct are written as multiplies
    // so that they issue on the multiply-add pipe instead of the integer ALU pipe.
    __device__ __forceinline__ uint32_t f(uint32_t r, uint32_t key) const {
        return __umulhi((r ^ key) * 0x9E3779B1u, up);
    }

    // Key of constraint x: four rounds of (L, R) -> (R, L ^ F(R)).
    __device__ __forceinline__ uint32_t enc(uint32_t x) const {
        uint32_t L = __umulhi(x, down), R = x - L * up, t;
        t = L ^ f(R, k0); L = R; R = t;
        t = L ^ f(R, k1); L = R; R = t;
        t = L ^ f(R, k2); L = R; R = t;
        t = L ^ f(R, k3); L = R; R = t;
        return L * up + R;
    }

    // Constraint with key x: rounds in reverse, (L, R) -> (R ^ F(L), L).
    __device__ __forceinline__ uint32_t dec(uint32_t x) const {
        uint32_t L = __umulhi(x, down), R = x - L * up, t;
        t = R ^ f(L, k3); R = L; L = t;
        t = R ^ f(L, k2); R = L; L = t;
        t = R ^ f(L, k1); R = L; L = t;
        t = R ^ f(L, k0); R = L; L = t;
        return L * up + R;
    }
};

// ---------------------------------------------------------------- reductions
// Order-preserving map of a float to a signed int (an involution): lets the warp
// min/max instructions (redux.sync) reduce float values.
__device__ __forceinline__ int float_key(float t) {
    int i = __float_as_int(t);
    return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float key_float(int k) {
    return __int_as_float(k ^ ((k >> 31) & 0x7fffffff));
}
__device__ __forceinline__ long long double_key(double t) {
    long long i = __double_as_longlong(t);
    return i ^ ((i >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ double key_double(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll));
}

// Warp-wide lexicographic min of (key, pos) -- 32-bit keys use redux.sync.
__device__ __forceinline__ void warp_min_pair(int& key, int& pos) {
    int kmin = __reduce_min_sync(kFull, key);
    pos = __reduce_min_sync(kFull, key == kmin ? pos : kNoPos);
    key = kmin;
}
// Warp-wide (max key, min pos among the max).
__device__ __forceinline__ void warp_max_pair(int& key, int& pos) {
    int kmax = __reduce_max_sync(kFull, key);
    pos = __reduce_min_sync(kFull, key == kmax ? pos : kNoPos);
    key = kmax;
}
__device__ __forceinline__ int warp_max_key(int key) { return __reduce_max_sync(kFull, key); }

// 64-bit keys: butterfly shuffles.
__device__ __forceinline__ void warp_min_pair(long long& key, int& pos) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        long long ok = __shfl_xor_sync(kFull, key, off);
        int op = __shfl_xor_sync(kFull, pos, off);
        if (ok < key || (ok == key && op < pos)) { key = ok; pos = op; }
    }
}
__device__ __forceinline__ void warp_max_pair(long long& key, int& pos) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        long long ok = __shfl_xor_sync(kFull, key, off);
        int op = __shfl_xor_sync(kFull, pos, off);
        if (ok > key || (ok == key && op < pos)) { key = ok; pos = op; }
    }
}

__device__ __forceinline__ long long warp_max_key(long long key) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const long long ok = __shfl_xor_sync(kFull, key, off);
        key = ok > key ? ok : key;
    }
    return key;
}

template <typename Real> struct KeyOf;
template <> struct KeyOf<float> {
    using type = int;
    __device__ static __forceinline__ int key(float t) { return float_key(t); }
    __device__ static __forceinline__ float val(int k) { return key_float(k); }
};
template <> struct KeyOf<double> {
    using type = long long;
    __device__ static __forceinline__ long long key(double t) { return double_key(t); }
    __device__ static __forceinline__ double val(long long k) { return key_double(k); }
};

template <typename Real> __device__ __forceinline__ Real real_inf();
template <> __device__ __forceinline__ float real_inf<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double real_inf<double>() { return __longlong_as_double(0x7ff0000000000000ll); }

template <typename Real> __device__ __forceinline__ Real real_div(Real a, Real b);
// FP32: the fast reciprocal-based division (about 2 ulp); FP64: IEEE division.
template <> __device__ __forceinline__ float real_div<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double real_div<double>(double a, double b) { return a / b; }

template <typename Real> __device__ __forceinline__ Real real_abs(Real a) { return a < Real(0) ? -a : a; }
template <typename Real> __device__ __forceinline__ Real real_max(Real a, Real b);
template <> __device__ __forceinline__ float real_max<float>(float a, float b) { return fmaxf(a, b); }
template <> __device__ __forceinline__ double real_max<double>(double a, double b) { return fmax(a, b); }

// Box side s (0..3) as a constraint g.x <= gb, at visit position s - 4:
//   0: x <= xmax   1: -x <= -xmin   2: y <= ymax   3: -y <= -ymin
template <typename Real>
__device__ __forceinline__ void box_side(const Params& P, int s, Real& gx, Real& gy, Real& gb) {
    gx = (s == 0) ? Real(1) : (s == 1) ? Real(-1) : Real(0);
    gy = (s == 2) ? Real(1) : (s == 3) ? Real(-1) : Real(0);
    gb = (s == 0) ? Real(P.xmax) : (s == 1) ? Real(-P.xmin) : (s == 2) ? Real(P.ymax) : Real(-P.ymin);
}

}  // namespace lp2d
