// hm_peak.cu -- measured FMA throughput of the current device, the
// denominator of the roofline fractions of the ALU-bound kernels.
//
// Every thread runs PK_CHAINS independent fused multiply-add chains, enough
// to cover the FMA latency at full occupancy; the grid is four full waves of
// resident CTAs. The result is written only under a condition that never
// holds, so the compiler keeps the work and the kernel stores nothing.
#include <cuda_runtime.h>

#include <algorithm>

#include "hm_internal.cuh"

namespace hm {

namespace {

constexpr int PK_NT = 256;
constexpr int PK_CHAINS = 8;

template <class T, int ITERS>
__global__ void __launch_bounds__(PK_NT) k_fma_peak(T b, T c, T* __restrict__ out)
{
    T a[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int k = 0; k < PK_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
    if (s == (T)-1) out[blockIdx.x] = s;
}

template <class T, int ITERS>
double measure()
{
    int occ = 0;
    HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_peak<T, ITERS>, PK_NT, 0));
    const int grid = std::max(occ, 1) * num_sms() * 4;
    cudaStream_t s = nullptr;
    HM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0;
    try {
        HM_CUDA(cudaEventCreate(&e0));
        HM_CUDA(cudaEventCreate(&e1));
        DevBuf<T> out((size_t)grid, s);
        const T b = (T)0.999999, c = (T)1e-6;
        k_fma_peak<T, ITERS><<<grid, PK_NT, 0, s>>>(b, c, out.p);   // warm-up
        note_launch();
        HM_LAUNCH("fma peak");
        for (int rep = 0; rep < 3; ++rep) {
            HM_CUDA(cudaEventRecord(e0, s));
            k_fma_peak<T, ITERS><<<grid, PK_NT, 0, s>>>(b, c, out.p);
            note_launch();
            HM_CUDA(cudaEventRecord(e1, s));
            HM_CUDA(cudaEventSynchronize(e1));
            HM_LAUNCH("fma peak");
            float ms = 0.f;
            HM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            const double fl = 2.0 * (double)grid * PK_NT * PK_CHAINS * ITERS;
            if (ms > 0.f) best = std::max(best, fl / (ms * 1e-3));
        }
        HM_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamDestroy(s);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    return best;
}

}  // namespace

double alu_peak(int precision)
{
    if (precision == HM_PREC_FP64) return measure<double, 512>();
    return measure<float, 8192>();
}

}  // namespace hm
