// hm_stream.cuh -- device pieces shared by the product kernels: the column
// chunk of the V^T x work items, the compensated float accumulator, bfloat16
// pair conversion, and the mbarrier / bulk-copy wrappers (inline PTX) with
// waits bounded by the global timer.
#pragma once
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>

namespace hm {
namespace {

constexpr int VCH = 256;          // columns per V^T x work item (8 per lane)

template <class R>
struct Acc;

template <>
struct Acc<double> {
    double s = 0.0;
    __device__ void add(double v) { s += v; }
    __device__ double value() const { return s; }
};

// Compensated float accumulation across contributions (Neumaier's variant of
// Kahan summation): the rounding error of every addition is kept in c.
template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ void add(float v)
    {
        float t = s + v;
        if (fabsf(s) >= fabsf(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    __device__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ float2 bf2(uint32_t u)
{
    __nv_bfloat162 h;
    memcpy(&h, &u, 4);
    return __bfloat1622float2(h);
}


// The producer's last waits, for copies it has issued, use at least this
// bound whatever the bound of the other waits: a CTA never exits while a
// bulk copy into its shared memory may be in flight.
constexpr uint64_t MBAR_DRAIN_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity to complete; false once the wait
// has lasted limit_ns (each try_wait itself suspends for a bounded time).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (int k = 0;; ++k) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(b)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (k == 0) t0 = global_ns();
        else if (global_ns() - t0 > limit_ns) return false;
    }
}
// Global -> shared bulk copy of bytes (a multiple of 16, both addresses
// 16-byte aligned), completing on mbarrier b.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* b)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(b))
        : "memory");
}

}  // namespace
}  // namespace hm
