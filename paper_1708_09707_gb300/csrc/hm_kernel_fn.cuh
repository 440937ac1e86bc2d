// hm_kernel_fn.cuh -- kernel functions phi(y, y') on Morton-ordered points.
//   Gaussian:    exp(-D2 * c),        c = 1 / l^2
//   Matern-3/2:  (1 + s) exp(-s),     s = sqrt(D2) * c,  c = sqrt(3) / l
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

template <int KERN>
__device__ __forceinline__ double phi(double D2, double c)
{
    if (KERN == HM_GAUSSIAN) return exp(-(D2 * c));
    double s = sqrt(D2) * c;
    return (1.0 + s) * exp(-s);
}

template <int KERN>
__device__ __forceinline__ float phi(float D2, float c)
{
    if (KERN == HM_GAUSSIAN) return expf(-(D2 * c));
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
