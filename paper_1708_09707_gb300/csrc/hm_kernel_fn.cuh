// hm_kernel_fn.cuh -- kernel functions phi(y, y') on Morton-ordered points.
//   Gaussian:    exp(-D2 * c),        c = 1 / l^2
//   Matern-3/2:  (1 + s) exp(-s),     s = sqrt(D2) * c,  c = sqrt(3) / l
//   Matern K_1:  s K_1(s), s = r / l, from t = s^2 / 4 = D2 * c, c = 1 / (4 l^2)
// (Sec. 6.2 model problem; l and the Matern order are the workloads' choice.)
// The double path loads double coordinates. The float path loads a hi/lo
// float split of every coordinate and forms each difference as
// (hi_a - hi_b) + (lo_a - lo_b), which keeps the difference accurate to about
// float precision relative to itself even when the points are far from the
// origin of the unit cube.
#pragma once

#include "hm_build.cuh"

namespace hm {

template <class R>
struct Pt;

template <>
struct Pt<double> {
    double x[3];
};

template <>
struct Pt<float> {
    float h[3], l[3];
};

__device__ __forceinline__ Pt<double> load_pt64(const DeviceCoords& X, int64_t row)
{
    Pt<double> p;
    p.x[0] = X.x64[0][row];
    p.x[1] = X.x64[1][row];
    p.x[2] = X.x64[2][row];
    return p;
}

__device__ __forceinline__ Pt<float> load_pt32(const DeviceCoords& X, int64_t row)
{
    Pt<float> p;
    const float* F = X.x32;
    const int64_t st = X.stride32;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p.h[i] = F[(2 * i) * st + row];
        p.l[i] = F[(2 * i + 1) * st + row];
    }
    return p;
}

template <class R>
__device__ __forceinline__ Pt<R> load_pt(const DeviceCoords& X, int64_t row);

template <>
__device__ __forceinline__ Pt<double> load_pt<double>(const DeviceCoords& X, int64_t row)
{
    return load_pt64(X, row);
}

template <>
__device__ __forceinline__ Pt<float> load_pt<float>(const DeviceCoords& X, int64_t row)
{
    return load_pt32(X, row);
}

__device__ __forceinline__ double dist2(const Pt<double>& a, const Pt<double>& b)
{
    double t0 = a.x[0] - b.x[0], t1 = a.x[1] - b.x[1], t2 = a.x[2] - b.x[2];
    return fma(t2, t2, fma(t1, t1, t0 * t0));
}

__device__ __forceinline__ float dist2(const Pt<float>& a, const Pt<float>& b)
{
    float t0 = (a.h[0] - b.h[0]) + (a.l[0] - b.l[0]);
    float t1 = (a.h[1] - b.h[1]) + (a.l[1] - b.l[1]);
    float t2 = (a.h[2] - b.h[2]) + (a.l[2] - b.l[2]);
    return fmaf(t2, t2, fmaf(t1, t1, t0 * t0));
}

// Matern kernel of order 1 (Sec. 6.2 with beta - d/2 = 1), normalised to
// phi(0) = 1: phi = s K_1(s), s = r / l, evaluated from t = s^2 / 4.
//  * t <= 1 (s <= 2): multiplying the ascending series of K_1 (Abramowitz
//    and Stegun 9.6.11) by s gives
//        s K_1(s) = 1 + t (ln(t) S0(t) - S1(t)),
//        S0 = sum_k c_k t^k,  S1 = sum_k (H_k + H_{k+1} - 2 gamma) c_k t^k,
//    with c_k = 1 / (k! (k+1)!), H_k the harmonic numbers and gamma Euler's
//    constant; Horner's rule over k <= 12 in double (c_13 < 2e-21) and
//    k <= 7 in float (c_8 < 7e-11). No square root is needed.
//  * t > 1: the integral K_1(s) = int_0^inf exp(-s cosh u) cosh u du (A&S
//    9.6.24) by the trapezoidal rule with step h. The integrand is entire and
//    even, so the rule's relative error is about exp(s (1 - cos a) - 2 pi a/h)
//    for any strip half-width a < pi/2: h = min(0.2, 0.6 / sqrt(s)) keeps it
//    below 1e-17 for every s > 2 (float: min(0.3, 1 / sqrt(s)), below 1e-8).
//    With E_j = cosh(jh) - 1 from E_{j+1} = 2 (1 + E_1) E_j - E_{j-1} + 2 E_1,
//    E_1 = 2 sinh^2(h/2) (no cancellation when jh is small),
//        s K_1(s) = s h e^{-s} (1/2 + sum_{j>=1} (1 + E_j) exp(-s E_j)),
//    summed while s E_j <= 42 (float: 20), at most 12 to 20 terms.
constexpr double K1_EULER = 0.57721566490153286061;

template <int K>
struct K1Coef {
    static constexpr double c = K1Coef<K - 1>::c / ((double)K * (double)(K + 1));
    static constexpr double h = K1Coef<K - 1>::h + 1.0 / K;     // H_K
    static constexpr double d = (2.0 * h + 1.0 / (K + 1) - 2.0 * K1_EULER) * c;
};
template <>
struct K1Coef<0> {
    static constexpr double c = 1.0;
    static constexpr double h = 0.0;
    static constexpr double d = 1.0 - 2.0 * K1_EULER;
};

// S0 and S1 by Horner's rule over k = K .. KMAX.
template <class R, int K, int KMAX>
struct K1Horner {
    __device__ __forceinline__ static void eval(R t, R& s0, R& s1)
    {
        K1Horner<R, K + 1, KMAX>::eval(t, s0, s1);
        s0 = fma(s0, t, (R)K1Coef<K>::c);
        s1 = fma(s1, t, (R)K1Coef<K>::d);
    }
};
template <class R, int KMAX>
struct K1Horner<R, KMAX, KMAX> {
    __device__ __forceinline__ static void eval(R, R& s0, R& s1)
    {
        s0 = (R)K1Coef<KMAX>::c;
        s1 = (R)K1Coef<KMAX>::d;
    }
};

__device__ __forceinline__ double matern_k1(double t)
{
    if (t <= 1.0) {
        if (t == 0.0) return 1.0;
        double s0, s1;
        K1Horner<double, 0, 12>::eval(t, s0, s1);
        return fma(t, fma(log(t), s0, -s1), 1.0);
    }
    const double s = 2.0 * sqrt(t);
    const double h = fmin(0.2, 0.6 / sqrt(s));
    const double sh = sinh(0.5 * h);
    const double e1 = 2.0 * sh * sh;
    const double c2 = 2.0 * (1.0 + e1);
    double em = 0.0, e = e1, acc = 0.5;
    for (int j = 1; j <= 64 && s * e <= 42.0; ++j) {
        acc = fma(1.0 + e, exp(-s * e), acc);
        const double en = fma(c2, e, 2.0 * e1 - em);
        em = e;
        e = en;
    }
    return s * h * exp(-s) * acc;
}

__device__ __forceinline__ float matern_k1(float t)
{
    if (t <= 1.f) {
        if (t == 0.f) return 1.f;
        float s0, s1;
        K1Horner<float, 0, 7>::eval(t, s0, s1);
        return fmaf(t, fmaf(logf(t), s0, -s1), 1.f);
    }
    const float s = 2.f * sqrtf(t);
    const float h = fminf(0.3f, 1.f / sqrtf(s));
    const float sh = sinhf(0.5f * h);
    const float e1 = 2.f * sh * sh;
    const float c2 = 2.f * (1.f + e1);
    float em = 0.f, e = e1, acc = 0.5f;
    for (int j = 1; j <= 32 && s * e <= 20.f; ++j) {
        acc = fmaf(1.f + e, expf(-s * e), acc);
        const float en = fmaf(c2, e, 2.f * e1 - em);
        em = e;
        e = en;
    }
    return s * h * expf(-s) * acc;
}

template <int KERN>
__device__ __forceinline__ double phi(double D2, double c)
{
    if (KERN == HM_GAUSSIAN) return exp(-(D2 * c));
    if (KERN == HM_MATERN_K1) return matern_k1(D2 * c);
    double s = sqrt(D2) * c;
    return (1.0 + s) * exp(-s);
}

template <int KERN>
__device__ __forceinline__ float phi(float D2, float c)
{
    if (KERN == HM_GAUSSIAN) return expf(-(D2 * c));
    if (KERN == HM_MATERN_K1) return matern_k1(D2 * c);
    float s = sqrtf(D2) * c;
    return (1.0f + s) * expf(-s);
}

template <class R>
__host__ __device__ __forceinline__ R kconst(const KernelParams& kp);

template <>
__host__ __device__ __forceinline__ double kconst<double>(const KernelParams& kp)
{
    return kp.c64;
}

template <>
__host__ __device__ __forceinline__ float kconst<float>(const KernelParams& kp)
{
    return kp.c32;
}

// Residual accumulator r = a - sum_l u_l v_l of the ACA cross updates: a
// fused multiply-add chain in the kernel's type. In float the chain's rounding
// is about sqrt(r) 2^-24 |a|, far below the accuracy asked of the
// approximation (eps >= 1e-6 relative to the block).
template <class R>
struct Resid {
    R s;
    __device__ __forceinline__ void init(R a) { s = a; }
    __device__ __forceinline__ void sub(R u, R v) { s = fma(-u, v, s); }
    __device__ __forceinline__ R value() const { return s; }
};

// Sum kept by one thread and combined over threads. In double a plain sum.
// In float a pair s + c: a thread adds its own terms plainly (it holds at
// most a few dozen, so its partial is accurate to about 1e-6 of itself),
// and the joins of partials across lanes, warps and CTAs are Knuth's TwoSum,
// whose exact rounding error is carried in c. The float kernels thus do no
// double arithmetic per entry (this GPU's double pipe runs at a small
// fraction of its float rate).
template <class R>
struct TSum;

template <>
struct TSum<double> {
    double s;
    __device__ __forceinline__ void init() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void set(double x) { s = x; }
    __device__ __forceinline__ void join(const TSum& o) { s += o.s; }
    __device__ __forceinline__ void shfl_join(int o) { s += __shfl_xor_sync(0xffffffffu, s, o); }
    __device__ __forceinline__ double value() const { return s; }
    __device__ __forceinline__ double rvalue() const { return s; }
};

template <>
struct TSum<float> {
    float s, c;
    __device__ __forceinline__ void init()
    {
        s = 0.f;
        c = 0.f;
    }
    __device__ __forceinline__ void add2(float x, float xc)
    {
        const float t = __fadd_rn(s, x);
        const float z = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));
        s = t;
        // (c + xc) + e: symmetric in the two operands, so a butterfly over a
        // warp leaves the same pair in every lane
        c = __fadd_rn(__fadd_rn(c, xc), e);
    }
    __device__ __forceinline__ void add(float x) { s += x; }
    __device__ __forceinline__ void set(float x)
    {
        s = x;
        c = 0.f;
    }
    __device__ __forceinline__ void join(const TSum& o) { add2(o.s, o.c); }
    __device__ __forceinline__ void shfl_join(int o)
    {
        const float os = __shfl_xor_sync(0xffffffffu, s, o);
        const float oc = __shfl_xor_sync(0xffffffffu, c, o);
        add2(os, oc);
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
    // the pair rounded to float (no double arithmetic)
    __device__ __forceinline__ float rvalue() const { return s + c; }
};

// Warp-wide helpers.
template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// argmax of (val, idx) with ties to the lower index.
template <class T>
__device__ __forceinline__ void warp_argmax(T& val, int& idx)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, val, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > val || (ov == val && oi < idx)) {
            val = ov;
            idx = oi;
        }
    }
}

}  // namespace hm
