// hm_near.cu -- batched evaluation of the dense (inadmissible) leaf blocks
// (Sec. 5.4.2). Every dense block is cut into the row tiles it covers and
// each slice is stored column-major with the tile's row count as leading
// dimension, in the product's gather order (tile-major); unlike the paper's
// stacked layout there is no zero padding to a common column count.
// Formats: double, float, bfloat16 hi/lo pair (hi = bf16(a), lo =
// bf16(a - hi), about 16 significant bits together; each column holds its hi
// entries, then its lo entries) or a single bf16.
#include "hm_kernel_fn.cuh"

#include <vector>

namespace hm {

namespace {

constexpr int NT = 128;

// One CTA per slice. Thread t owns the row pair (2p, 2p + 1), p = t mod
// (ld / 2), keeps both row points in registers and walks the columns
// t / (ld / 2), stepping by NT / (ld / 2); a warp thus covers consecutive row
// pairs of one column and stores them as one contiguous vector line. Slices
// taller than 2 NT rows are done in row passes of 2 NT.
template <int KERN, int FMT>
__global__ void __launch_bounds__(NT)
k_near(KernelParams kp, DeviceCoords X, const Blk* __restrict__ blk, const int2* __restrict__ ent,
       const int32_t* __restrict__ etile, const int32_t* __restrict__ tile_m,
       const DnDesc* __restrict__ desc, int64_t ne, void* __restrict__ store)
{
    const int64_t e = blockIdx.x;
    if (e >= ne) return;
    const int2 en = ent[e];
    const Blk B = blk[en.x];
    const int rows = tile_m[etile[e]];
    const int ld = slice_ld(rows);
    const int64_t r0 = B.row0 + en.y;
    const int n = B.n;
    const int64_t o = desc[e].noff;
    for (int pr0 = 0; pr0 < ld / 2; pr0 += NT) {
        const int npair = min(NT, ld / 2 - pr0);
        const int cstep = NT / npair;
        const int t = threadIdx.x;
        if (t >= cstep * npair) continue;
        const int i = 2 * (pr0 + t % npair);      // first row of the pair
        const bool v0 = i < rows, v1 = i + 1 < rows;
        // the pair's points (padding rows load the last real row)
        const int64_t ra = r0 + min(i, rows - 1), rb = r0 + min(i + 1, rows - 1);
        Pt<double> pa64, pb64;
        Pt<float> pa32, pb32;
        if (FMT == HM_NEAR_FP64) {
            pa64 = load_pt64(X, ra);
            pb64 = load_pt64(X, rb);
        } else {
            pa32 = load_pt32(X, ra);
            pb32 = load_pt32(X, rb);
        }
        for (int j = t / npair; j < n; j += cstep) {
            const int64_t q = (int64_t)j * ld + i;
            if (FMT == HM_NEAR_FP64) {
                const Pt<double> pc = load_pt64(X, B.col0 + j);
                double2 v;
                v.x = v0 ? phi<KERN>(dist2(pa64, pc), kp.c64) : 0.0;
                v.y = v1 ? phi<KERN>(dist2(pb64, pc), kp.c64) : 0.0;
                *reinterpret_cast<double2*>(static_cast<double*>(store) + o + q) = v;
            } else {
                // float kernel evaluation from the hi/lo coordinate split
                const Pt<float> pc = load_pt32(X, B.col0 + j);
                const float a = v0 ? phi<KERN>(dist2(pa32, pc), kp.c32) : 0.f;
                const float b = v1 ? phi<KERN>(dist2(pb32, pc), kp.c32) : 0.f;
                if (FMT == HM_NEAR_FP32) {
                    *reinterpret_cast<float2*>(static_cast<float*>(store) + o + q) = make_float2(a, b);
                } else if (FMT == HM_NEAR_BF16X2) {
                    // column j: hi entries at 2 j ld, lo entries at 2 j ld + ld
                    __nv_bfloat16* S = static_cast<__nv_bfloat16*>(store) + 2 * o + q + (int64_t)j * ld;
                    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                    const float2 hf = __bfloat1622float2(h);
                    *reinterpret_cast<__nv_bfloat162*>(S) = h;
                    *reinterpret_cast<__nv_bfloat162*>(S + ld) = __floats2bfloat162_rn(a - hf.x, b - hf.y);
                } else {
                    *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(store) + o + q) =
                        __floats2bfloat162_rn(a, b);
                }
            }
        }
    }
}

template <int KERN>
void launch(int fmt, const KernelParams& kp, const DeviceCoords& X, const Blk* blk,
            const int2* ent, const int32_t* etile, const int32_t* tile_m, const DnDesc* desc,
            int64_t n, void* store, cudaStream_t s)
{
    const unsigned g = (unsigned)n;
    switch (fmt) {
    case HM_NEAR_FP64: k_near<KERN, HM_NEAR_FP64><<<g, NT, 0, s>>>(kp, X, blk, ent, etile, tile_m, desc, n, store); note_launch(); break;
    case HM_NEAR_FP32: k_near<KERN, HM_NEAR_FP32><<<g, NT, 0, s>>>(kp, X, blk, ent, etile, tile_m, desc, n, store); note_launch(); break;
    case HM_NEAR_BF16X2: k_near<KERN, HM_NEAR_BF16X2><<<g, NT, 0, s>>>(kp, X, blk, ent, etile, tile_m, desc, n, store); note_launch(); break;
    default: k_near<KERN, HM_NEAR_BF16><<<g, NT, 0, s>>>(kp, X, blk, ent, etile, tile_m, desc, n, store); note_launch(); break;
    }
}

// Sum of phi^2 over the entries of each dense leaf (one warp per leaf, the
// float kernel functions of the mixed path); out[b] in double.
template <int KERN>
__global__ void k_dense_fro2(KernelParams kp, DeviceCoords X, const Blk* __restrict__ blk,
                             int64_t n, double* __restrict__ out)
{
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= n) return;
    const Blk B = blk[b];
    const float c = kconst<float>(kp);
    double s = 0.0;
    for (int i = 0; i < B.m; ++i) {
        const Pt<float> pi = load_pt<float>(X, B.row0 + i);
        float si = 0.f;
        for (int j = lane; j < B.n; j += 32) {
            const float v = phi<KERN>(dist2(pi, load_pt<float>(X, B.col0 + j)), c);
            si = fmaf(v, v, si);
        }
        s += (double)si;
    }
    s = warp_sum(s);
    if (lane == 0) out[b] = s;
}

}  // namespace

double dense_fro2(const KernelParams& kp, const DeviceCoords& X, const Blk* blk, int64_t n,
                  cudaStream_t s)
{
    if (n <= 0) return 0.0;
    DevBuf<double> part(n, s);
    const unsigned g = (unsigned)ceil_div(n * 32, (int64_t)256);
    if (kp.kernel == HM_GAUSSIAN)
        k_dense_fro2<HM_GAUSSIAN><<<g, 256, 0, s>>>(kp, X, blk, n, part.p);
    else if (kp.kernel == HM_MATERN32)
        k_dense_fro2<HM_MATERN32><<<g, 256, 0, s>>>(kp, X, blk, n, part.p);
    else
        k_dense_fro2<HM_MATERN_K1><<<g, 256, 0, s>>>(kp, X, blk, n, part.p);
    note_launch();
    HM_LAUNCH("dense leaf norms");
    std::vector<double> h(n);
    HM_CUDA(cudaMemcpyAsync(h.data(), part.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    double sum = 0.0;          // in leaf order: the same value on every run
    for (int64_t b = 0; b < n; ++b) sum += h[b];
    return sum;
}

size_t near_entry_bytes(int fmt)
{
    switch (fmt) {
    case HM_NEAR_FP64: return 8;
    case HM_NEAR_FP32: return 4;
    case HM_NEAR_BF16X2: return 4;
    default: return 2;
    }
}

void near_assemble(int fmt, const KernelParams& kp, const DeviceCoords& X, const Blk* blk,
                   const int2* ent, const int32_t* etile, const int32_t* tile_m,
                   const DnDesc* desc, int64_t n, void* store, cudaStream_t s)
{
    if (n <= 0) return;
    if (n > 0x7fffffffll) fail(HM_EOVERFLOW, "too many dense slices for one launch");
    if (kp.kernel == HM_GAUSSIAN) launch<HM_GAUSSIAN>(fmt, kp, X, blk, ent, etile, tile_m, desc, n, store, s);
    else if (kp.kernel == HM_MATERN32) launch<HM_MATERN32>(fmt, kp, X, blk, ent, etile, tile_m, desc, n, store, s);
    else launch<HM_MATERN_K1>(fmt, kp, X, blk, ent, etile, tile_m, desc, n, store, s);
    HM_LAUNCH("near field");
}

}  // namespace hm
