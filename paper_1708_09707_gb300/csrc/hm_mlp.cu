// hm_mlp.cu -- learned rank model (not in the paper): features of admissible
// blocks, MLP 8 -> 64 -> 64 -> 1 forward, mean-squared-error gradient and Adam,
// all FP32 on the device, plus the rank prediction and misprediction re-run
// used by the build.
//
//   features f = [d/3, log2|tau|/16, log2|sigma|/16, log2(1 + diam_tau/l),
//                 log2(1 + diam_sigma/l), log2(1 + dist/l), -log10(eps)/8, kernel]
//   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), yhat = W3 h2 + b3,
//   target log2(1 + rank); the build reserves ceil(1.25 (2^yhat - 1) + 2)
//   columns (clamped to [1, min(k_cap, m, n)]).
// Gradients are summed per CTA over a tile of 64 samples and the per-CTA
// partials are added in CTA order, so the result is deterministic.
#include <cmath>

#include "hm_handle.cuh"
#include "hm_mlp.cuh"

namespace hm {

namespace {

constexpr int NT = 256;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_H * MLP_F;
constexpr int OFF_W2 = OFF_B1 + MLP_H;
constexpr int OFF_B2 = OFF_W2 + MLP_H * MLP_H;
constexpr int OFF_W3 = OFF_B2 + MLP_H;
constexpr int OFF_B3 = OFF_W3 + MLP_H;
constexpr int GS = 64;   // samples per CTA in the gradient kernel

inline unsigned grid_for(int64_t n) { return (unsigned)ceil_div(n, NT); }

__global__ void __launch_bounds__(NT)
k_mlp_fwd(const float* __restrict__ theta, const float* __restrict__ F, int64_t n,
          float* __restrict__ out)
{
    __shared__ float th[MLP_NPARAM];
    for (int p = threadIdx.x; p < MLP_NPARAM; p += NT) th[p] = theta[p];
    __syncthreads();
    int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (s >= n) return;
    float f[MLP_F];
#pragma unroll
    for (int i = 0; i < MLP_F; ++i) f[i] = F[s * MLP_F + i];
    float h1[MLP_H];
#pragma unroll
    for (int o = 0; o < MLP_H; ++o) {
        float a = th[OFF_B1 + o];
#pragma unroll
        for (int i = 0; i < MLP_F; ++i) a = fmaf(th[OFF_W1 + o * MLP_F + i], f[i], a);
        h1[o] = fmaxf(a, 0.f);
    }
    float y = th[OFF_B3];
    for (int o = 0; o < MLP_H; ++o) {
        float a = th[OFF_B2 + o];
#pragma unroll
        for (int i = 0; i < MLP_H; ++i) a = fmaf(th[OFF_W2 + o * MLP_H + i], h1[i], a);
        y = fmaf(th[OFF_W3 + o], fmaxf(a, 0.f), y);
    }
    out[s] = y;
}

struct GradSmem {
    float th[MLP_NPARAM];
    float F[GS][MLP_F];
    float H1[GS][MLP_H];
    float H2[GS][MLP_H];
    float D2[GS][MLP_H];
    float D1[GS][MLP_H];
    float dy[GS];
    float e2[GS];
};

__global__ void __launch_bounds__(NT)
k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ F,
           const float* __restrict__ target, int64_t n, float* __restrict__ part,
           float* __restrict__ lpart)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    GradSmem& S = *reinterpret_cast<GradSmem*>(smraw);
    const int tid = threadIdx.x;
    for (int p = tid; p < MLP_NPARAM; p += NT) S.th[p] = theta[p];
    const int64_t s0 = (int64_t)blockIdx.x * GS;
    const int ns = (n - s0) < GS ? (int)(n - s0) : GS;
    for (int e = tid; e < GS * MLP_F; e += NT) {
        int s = e / MLP_F, i = e % MLP_F;
        S.F[s][i] = s < ns ? F[(s0 + s) * MLP_F + i] : 0.f;
    }
    __syncthreads();
    // forward, one thread per sample (the other threads wait)
    if (tid < GS) {
        const int s = tid;
        float y = S.th[OFF_B3];
        for (int o = 0; o < MLP_H; ++o) {
            float a = S.th[OFF_B1 + o];
            for (int i = 0; i < MLP_F; ++i) a = fmaf(S.th[OFF_W1 + o * MLP_F + i], S.F[s][i], a);
            S.H1[s][o] = fmaxf(a, 0.f);
        }
        for (int o = 0; o < MLP_H; ++o) {
            float a = S.th[OFF_B2 + o];
            for (int i = 0; i < MLP_H; ++i) a = fmaf(S.th[OFF_W2 + o * MLP_H + i], S.H1[s][i], a);
            const float h = fmaxf(a, 0.f);
            S.H2[s][o] = h;
            y = fmaf(S.th[OFF_W3 + o], h, y);
        }
        const float e = s < ns ? y - target[s0 + s] : 0.f;
        S.dy[s] = 2.f * e / (float)n;
        S.e2[s] = e * e;
    }
    __syncthreads();
    // back through layer 3 and the second ReLU
    for (int e = tid; e < GS * MLP_H; e += NT) {
        int s = e / MLP_H, o = e % MLP_H;
        S.D2[s][o] = S.H2[s][o] > 0.f ? S.dy[s] * S.th[OFF_W3 + o] : 0.f;
    }
    __syncthreads();
    // back through layer 2 and the first ReLU
    for (int e = tid; e < GS * MLP_H; e += NT) {
        int s = e / MLP_H, i = e % MLP_H;
        float a = 0.f;
        for (int o = 0; o < MLP_H; ++o) a = fmaf(S.th[OFF_W2 + o * MLP_H + i], S.D2[s][o], a);
        S.D1[s][i] = S.H1[s][i] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // parameter gradients summed over this CTA's samples in sample order
    float* out = part + (int64_t)blockIdx.x * MLP_NPARAM;
    for (int p = tid; p < MLP_NPARAM; p += NT) {
        float g = 0.f;
        if (p < OFF_B1) {
            int o = p / MLP_F, i = p % MLP_F;
            for (int s = 0; s < GS; ++s) g = fmaf(S.D1[s][o], S.F[s][i], g);
        } else if (p < OFF_W2) {
            int o = p - OFF_B1;
            for (int s = 0; s < GS; ++s) g += S.D1[s][o];
        } else if (p < OFF_B2) {
            int o = (p - OFF_W2) / MLP_H, i = (p - OFF_W2) % MLP_H;
            for (int s = 0; s < GS; ++s) g = fmaf(S.D2[s][o], S.H1[s][i], g);
        } else if (p < OFF_W3) {
            int o = p - OFF_B2;
            for (int s = 0; s < GS; ++s) g += S.D2[s][o];
        } else if (p < OFF_B3) {
            int o = p - OFF_W3;
            for (int s = 0; s < GS; ++s) g = fmaf(S.dy[s], S.H2[s][o], g);
        } else {
            for (int s = 0; s < GS; ++s) g += S.dy[s];
        }
        out[p] = g;
    }
    if (tid == 0) {
        float l = 0.f;
        for (int s = 0; s < GS; ++s) l += S.e2[s];
        lpart[blockIdx.x] = l;
    }
}

__global__ void k_mlp_sum(const float* __restrict__ part, const float* __restrict__ lpart,
                          int nparts, int64_t n, float* __restrict__ grad, float* __restrict__ loss)
{
    int p = blockIdx.x * NT + threadIdx.x;
    if (p < MLP_NPARAM) {
        float g = 0.f;
        for (int c = 0; c < nparts; ++c) g += part[(int64_t)c * MLP_NPARAM + p];
        grad[p] = g;
    }
    if (p == 0 && loss) {
        double l = 0.0;
        for (int c = 0; c < nparts; ++c) l += lpart[c];
        *loss = (float)(l / (double)n);
    }
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    int p = blockIdx.x * NT + threadIdx.x;
    if (p >= n) return;
    float gi = g[p];
    float mi = b1 * m[p] + (1.f - b1) * gi;
    float vi = b2 * v[p] + (1.f - b2) * gi * gi;
    m[p] = mi;
    v[p] = vi;
    th[p] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Features of every admissible block (and the log2(1 + rank) target).
__global__ void k_features(const int2* __restrict__ pairs, const int32_t* __restrict__ bset,
                           int64_t n, const int64_t* __restrict__ set_node0,
                           const int32_t* __restrict__ set_d, const double* __restrict__ bmin,
                           const double* __restrict__ bmax, const int32_t* __restrict__ lo,
                           const int32_t* __restrict__ hi, double ell, double aca_eps, int kernel,
                           const int32_t* __restrict__ rank, float* __restrict__ F,
                           float* __restrict__ target, const uint32_t* __restrict__ ids)
{
    int64_t r = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (r >= n) return;
    const int64_t b = ids ? (int64_t)ids[r] : r;   // the block of feature row r
    const int q = bset[b];
    const int64_t base = set_node0[q];
    const int64_t t = base + pairs[b].x, s = base + pairs[b].y;
    double Dt = 0.0, Ds = 0.0, G2 = 0.0;
    for (int i = 0; i < 3; ++i) {
        double et = bmax[t * 3 + i] - bmin[t * 3 + i];
        double es = bmax[s * 3 + i] - bmin[s * 3 + i];
        Dt += et * et;
        Ds += es * es;
        double g1 = fmax(0.0, bmin[t * 3 + i] - bmax[s * 3 + i]);
        double g2 = fmax(0.0, bmin[s * 3 + i] - bmax[t * 3 + i]);
        G2 += g1 * g1 + g2 * g2;
    }
    float* f = F + r * MLP_F;
    f[0] = (float)(set_d[q] / 3.0);
    f[1] = (float)(log2((double)(hi[t] - lo[t])) / 16.0);
    f[2] = (float)(log2((double)(hi[s] - lo[s])) / 16.0);
    f[3] = (float)log2(1.0 + sqrt(Dt) / ell);
    f[4] = (float)log2(1.0 + sqrt(Ds) / ell);
    f[5] = (float)log2(1.0 + sqrt(G2) / ell);
    f[6] = (float)(-log10(aca_eps) / 8.0);
    f[7] = (float)kernel;
    if (target && rank) target[r] = (float)log2(1.0 + (double)rank[b]);
}

__global__ void k_pred_to_rank(const float* __restrict__ yhat, int64_t n,
                               const uint32_t* __restrict__ ids, int32_t* __restrict__ k)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    float r = ceilf(1.25f * (exp2f(fminf(yhat[b], 8.f)) - 1.f) + 2.f);
    k[ids ? (int64_t)ids[b] : b] = (int32_t)fmaxf(r, 1.f);
}

__global__ void k_flag_mispred(const int32_t* __restrict__ flags, int64_t n,
                               int64_t* __restrict__ f)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b < n) f[b] = (flags[b] & 1) ? 1 : 0;
}

__global__ void k_emit_ids(const int64_t* __restrict__ f, const int64_t* __restrict__ off,
                           int64_t n, uint32_t* __restrict__ ids)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b < n && f[b]) ids[off[b]] = (uint32_t)b;
}

// Features of the admissible blocks ids[0..n) (all blocks when ids is null),
// one row per listed block.
void features(hm_handle_s& h, float* F, float* target, cudaStream_t s,
              const uint32_t* ids = nullptr, int64_t nids = -1)
{
    const int64_t n = ids ? nids : h.n_adm;
    if (n <= 0) return;
    std::vector<int64_t> n0(h.sets.size());
    std::vector<int32_t> dd(h.sets.size());
    for (size_t q = 0; q < h.sets.size(); ++q) {
        n0[q] = h.sets[q].node0;
        dd[q] = h.sets[q].d;
    }
    DevBuf<int64_t> sn0(n0.size(), s);
    DevBuf<int32_t> sd(dd.size(), s);
    copy_in(sn0.p, n0.data(), n0.size() * sizeof(int64_t), s);
    copy_in(sd.p, dd.data(), dd.size() * sizeof(int32_t), s);
    k_features<<<grid_for(n), NT, 0, s>>>(h.adm_pairs.p, h.adm_set.p, n, sn0.p, sd.p, h.bmin.p,
                                         h.bmax.p, h.node_lo.p, h.node_hi.p, h.ell, h.aca_eps,
                                         h.kernel, target ? h.rank.p : nullptr, F, target, ids); note_launch();
    HM_LAUNCH("features");
    HM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

void mlp_forward(const float* theta, const float* F, int64_t n, float* out, cudaStream_t s)
{
    if (n <= 0) return;
    k_mlp_fwd<<<grid_for(n), NT, 0, s>>>(theta, F, n, out); note_launch();
    HM_LAUNCH("mlp forward");
}

void mlp_loss_grad(const float* theta, const float* F, const float* target, int64_t n,
                   float* grad, float* loss, cudaStream_t s)
{
    if (n <= 0) fail(HM_EINVAL, "empty training batch");
    const int nparts = (int)ceil_div(n, GS);
    DevBuf<float> part((size_t)nparts * MLP_NPARAM, s), lpart(nparts, s);
    const int smem = (int)sizeof(GradSmem);
    HM_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_mlp_grad<<<nparts, NT, smem, s>>>(theta, F, target, n, part.p, lpart.p); note_launch();
    k_mlp_sum<<<grid_for(MLP_NPARAM), NT, 0, s>>>(part.p, lpart.p, nparts, n, grad, loss); note_launch();
    HM_LAUNCH("mlp grad");
}

void mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t t, float lr, float b1,
              float b2, float eps, cudaStream_t s)
{
    if (t < 1) fail(HM_EINVAL, "Adam step count must be >= 1");
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)t));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)t));
    k_adam<<<grid_for(MLP_NPARAM), NT, 0, s>>>(theta, grad, m, v, MLP_NPARAM, lr, b1, b2, eps, c1, c2); note_launch();
    HM_LAUNCH("adam");
}

void predict_ranks(hm_handle_s& h, int32_t* kpred, const uint32_t* ids, int64_t nids)
{
    cudaStream_t s = h.stream;
    const int64_t n = ids ? nids : h.n_adm;
    if (n <= 0) return;
    if (!h.opt.rank_model_theta) fail(HM_EINVAL, "rank_model set without rank_model_theta");
    DevBuf<float> th(MLP_NPARAM, s), F(n * MLP_F, s), y(n, s);
    copy_in(th.p, h.opt.rank_model_theta, MLP_NPARAM * sizeof(float), s);
    features(h, F.p, nullptr, s, ids, n);
    mlp_forward(th.p, F.p, n, y.p, s);
    k_pred_to_rank<<<grid_for(n), NT, 0, s>>>(y.p, n, ids, kpred); note_launch();
    HM_LAUNCH("predict ranks");
}

void rerun_mispredicted(hm_handle_s& h)
{
    cudaStream_t s = h.stream;
    const int64_t n = h.n_adm;
    if (n == 0) return;
    DevBuf<int64_t> f(n, s), off(n + 1, s);
    k_flag_mispred<<<grid_for(n), NT, 0, s>>>(h.flags.p, n, f.p); note_launch();
    scan_exclusive_i64(f.p, off.p, n, off.p + n, s);
    int64_t cnt = 0;
    HM_CUDA(cudaMemcpyAsync(&cnt, off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    h.stats.n_mispredicted = cnt;
    if (cnt == 0) return;
    DevBuf<uint32_t> ids(cnt, s);
    k_emit_ids<<<grid_for(n), NT, 0, s>>>(f.p, off.p, n, ids.p); note_launch();
    HM_LAUNCH("mispredicted ids");
    compress(h, ids.p, cnt, nullptr, true);
}

}  // namespace hm

using namespace hm;

extern "C" {

int hm_block_features(hm_handle h, float* feats, float* target)
{
    set_error("");
    try {
        if (!h || !feats) fail(HM_EINVAL, "null argument");
        cudaStream_t s = h->stream;
        const int64_t n = h->n_adm;
        if (n == 0) return HM_OK;
        DevBuf<float> F(n * MLP_F, s), T(n, s);
        features(*h, F.p, T.p, s);
        copy_out(feats, F.p, n * MLP_F * sizeof(float), s);
        if (target) copy_out(target, T.p, n * sizeof(float), s);
        HM_CUDA(cudaStreamSynchronize(s));
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_mlp_forward(const float* theta, const float* F, int64_t n, float* out, void* stream)
{
    set_error("");
    try {
        if (!theta || !F || !out || n < 0) fail(HM_EINVAL, "bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        const bool dev = is_device_ptr(F) && is_device_ptr(out) && is_device_ptr(theta);
        if (dev) {
            mlp_forward(theta, F, n, out, s);
            return HM_OK;
        }
        DevBuf<float> th(MLP_NPARAM, s), f(std::max<int64_t>(n, 1) * MLP_F, s), o(std::max<int64_t>(n, 1), s);
        copy_in(th.p, theta, MLP_NPARAM * sizeof(float), s);
        copy_in(f.p, F, n * MLP_F * sizeof(float), s);
        mlp_forward(th.p, f.p, n, o.p, s);
        copy_out(out, o.p, n * sizeof(float), s);
        HM_CUDA(cudaStreamSynchronize(s));
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_mlp_loss_grad(const float* theta, const float* F, const float* target, int64_t n,
                     float* grad, float* loss, void* stream)
{
    set_error("");
    try {
        if (!theta || !F || !target || !grad || n < 1) fail(HM_EINVAL, "bad arguments");
        mlp_loss_grad(theta, F, target, n, grad, loss, (cudaStream_t)stream);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t t, float lr, float b1,
                float b2, float eps, void* stream)
{
    set_error("");
    try {
        if (!theta || !grad || !m || !v) fail(HM_EINVAL, "null argument");
        mlp_adam(theta, grad, m, v, t, lr, b1, b2, eps, (cudaStream_t)stream);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

}  // extern "C"
