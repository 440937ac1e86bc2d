// hm_near.cu -- batched evaluation of the dense (inadmissible) leaf blocks
// (Sec. 5.4.2). Every dense block is cut into the row tiles it covers and
// each slice is stored column-major with the tile's row count as leading
// dimension, in the product's gather order (tile-major); unlike the paper's
// stacked layout there is no zero padding to a common column count.
// Formats: double, float, bfloat16 hi/lo pair (two planes: hi = bf16(a),
// lo = bf16(a - hi), about 16 significant bits together) or a single bf16.
#include "hm_kernel_fn.cuh"

namespace hm {

namespace {

constexpr int NT = 128;

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
    const int ld = rows + (rows & 1);   // even leading dimension (zero pad row)
    const int64_t r0 = B.row0 + en.y;
    const int64_t mn = (int64_t)ld * B.n;
    const int64_t o = desc[e].noff;
    for (int64_t q = threadIdx.x; q < mn; q += NT) {
        const int i = (int)(q % ld), j = (int)(q / ld);
        const bool pad = i >= rows;
        if (FMT == HM_NEAR_FP64) {
            double v = pad ? 0.0 : phi<KERN>(dist2(load_pt64(X, r0 + i), load_pt64(X, B.col0 + j)), kp.c64);
            static_cast<double*>(store)[o + q] = v;
        } else {
            // float kernel evaluation from the hi/lo coordinate split
            float v = pad ? 0.f : phi<KERN>(dist2(load_pt32(X, r0 + i), load_pt32(X, B.col0 + j)), kp.c32);
            if (FMT == HM_NEAR_FP32) {
                static_cast<float*>(store)[o + q] = v;
            } else if (FMT == HM_NEAR_BF16X2) {
                __nv_bfloat16* S = static_cast<__nv_bfloat16*>(store) + 2 * o;
                __nv_bfloat16 h = __float2bfloat16_rn(v);
                S[q] = h;
                S[mn + q] = __float2bfloat16_rn(v - __bfloat162float(h));
            } else {
                static_cast<__nv_bfloat16*>(store)[o + q] = __float2bfloat16_rn(v);
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

}  // namespace

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
    else launch<HM_MATERN32>(fmt, kp, X, blk, ent, etile, tile_m, desc, n, store, s);
    HM_LAUNCH("near field");
}

}  // namespace hm
