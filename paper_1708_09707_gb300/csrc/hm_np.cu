// hm_np.cu -- kernels of the product that stores nothing but the block
// structure (the paper's non-precomputed mode, Sec. 5.4 with the factors and
// the dense blocks recomputed for every product): per pass of admissible
// leaves the ACA factors are rebuilt in a bounded scratch area and applied at
// once, and the dense leaves are evaluated inside the product.
//
// Determinism: every row of y is one running sum in double, fed in a fixed
// order: the admissible leaves of the row's tile in block order (the passes
// take consecutive block ranges), then its dense leaves in block order.
#include "hm_kernel_fn.cuh"
#include "hm_stream.cuh"

namespace hm {

namespace {

constexpr int NT = 256;
inline unsigned grid_for(int64_t n, int nt = NT) { return (unsigned)ceil_div(n, nt); }

template <class R>
__global__ void k_np_gather_x(const double* __restrict__ x, const int64_t* __restrict__ perm,
                              int64_t N, R* __restrict__ xm)
{
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i < N) xm[i] = (R)x[perm[i]];
}

// t_b = V_b^T x|sigma for the blocks b0 .. b0 + nb - 1: one warp per block,
// lane j sums the columns j, j + 32, ... of every factor row l, the lane sums
// meet in the xor butterfly. t_b starts at t + (b - b0) kcap.
template <class R>
__global__ void k_np_vtx(const Blk* __restrict__ blk, const int32_t* __restrict__ rank,
                         const uint64_t* __restrict__ Vptr, int64_t b0, int64_t nb,
                         const R* __restrict__ xm, R* __restrict__ t, int kcap)
{
    const int64_t w = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nb) return;
    const int64_t b = b0 + w;
    const Blk B = blk[b];
    const int k = rank[b];
    const int n = B.n;
    const R* __restrict__ V = reinterpret_cast<const R*>(Vptr[b]);
    const R* __restrict__ xs = xm + B.col0;
    R* out = t + w * kcap;
    for (int l = 0; l < k; ++l) {
        const R* Vl = V + (int64_t)l * n;
        R s = R(0);
        for (int j = lane; j < n; j += 32) s = fma(__ldcs(Vl + j), xs[j], s);
        s = warp_sum(s);
        if (lane == 0) out[l] = s;
    }
}

// y_m += U_b t_b over the admissible leaves b0 <= b < b1 of every row tile,
// in block order; one warp per tile, lane i takes rows i, i + 32, ...
template <class R>
__global__ void k_np_apply(const int64_t* __restrict__ lr_ptr, const int2* __restrict__ lr_ent,
                           const Blk* __restrict__ blk, const int32_t* __restrict__ rank,
                           const uint64_t* __restrict__ Uptr, const int64_t* __restrict__ tile_row0,
                           const int32_t* __restrict__ tile_m, int64_t n_tiles, int64_t b0,
                           int64_t b1, const R* __restrict__ t, int kcap, double* __restrict__ yacc)
{
    const int64_t tile = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= n_tiles) return;
    const int64_t r0 = tile_row0[tile];
    const int mt = tile_m[tile];
    const int64_t e0 = lr_ptr[tile], e1 = lr_ptr[tile + 1];
    for (int i = lane; i < mt; i += 32) {
        double yv = yacc[r0 + i];
        for (int64_t e = e0; e < e1; ++e) {
            const int2 en = lr_ent[e];
            if (en.x < b0) continue;
            if (en.x >= b1) break;   // entries ascend by block
            const int k = rank[en.x];
            const int m = blk[en.x].m;
            const R* __restrict__ U = reinterpret_cast<const R*>(Uptr[en.x]) + en.y + i;
            const R* __restrict__ tb = t + (int64_t)(en.x - b0) * kcap;
            R c = R(0);
            for (int l = 0; l < k; ++l) c = fma(U[(int64_t)l * m], tb[l], c);
            yv += (double)c;
        }
        yacc[r0 + i] = yv;
    }
}

// y_m += A_b x|sigma over the dense leaves of every row tile, the entries
// phi(y_i, y_j) evaluated on the fly (the same kernel functions as the stored
// near field); one warp per tile, lane i takes rows i, i + 32, ... Each leaf's
// plain sum goes into a compensated accumulator (float) or a double sum.
template <class R, int KERN>
__global__ void k_np_near(KernelParams kp, DeviceCoords X, const Blk* __restrict__ dblk,
                          const int64_t* __restrict__ dn_ptr, const int2* __restrict__ dn_ent,
                          const int64_t* __restrict__ tile_row0, const int32_t* __restrict__ tile_m,
                          int64_t n_tiles, const R* __restrict__ xm, double* __restrict__ yacc)
{
    const int64_t tile = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= n_tiles) return;
    const int64_t r0 = tile_row0[tile];
    const int mt = tile_m[tile];
    const int64_t e0 = dn_ptr[tile], e1 = dn_ptr[tile + 1];
    const R c = kconst<R>(kp);
    for (int i = lane; i < mt; i += 32) {
        const Pt<R> p = load_pt<R>(X, r0 + i);
        Acc<R> acc;
        for (int64_t e = e0; e < e1; ++e) {
            const Blk B = dblk[dn_ent[e].x];
            R s = R(0);
            for (int j = 0; j < B.n; ++j) {
                const Pt<R> q = load_pt<R>(X, B.col0 + j);
                s = fma(phi<KERN>(dist2(p, q), c), xm[B.col0 + j], s);
            }
            acc.add(s);
        }
        yacc[r0 + i] += acc.value();
    }
}

__global__ void k_np_finish(const int64_t* __restrict__ perm, const double* __restrict__ sig_row,
                            double sigma2, int64_t N, const double* __restrict__ yacc,
                            const double* __restrict__ x, double* __restrict__ y, int accumulate)
{
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i >= N) return;
    const int64_t dst = perm[i];
    const double sg = sig_row ? sig_row[i] : sigma2;
    const double v = yacc[i] + sg * x[dst];
    y[dst] = accumulate ? y[dst] + v : v;
}

}  // namespace

void np_gather_x(int precision, const double* x, const int64_t* perm, int64_t N, void* xm,
                 cudaStream_t s)
{
    if (N <= 0) return;
    if (precision == HM_PREC_FP64)
        k_np_gather_x<double><<<grid_for(N), NT, 0, s>>>(x, perm, N, static_cast<double*>(xm));
    else
        k_np_gather_x<float><<<grid_for(N), NT, 0, s>>>(x, perm, N, static_cast<float*>(xm));
    note_launch();
    HM_LAUNCH("np gather x");
}

void np_lowrank(int precision, const Blk* ablk, const int32_t* rank, const uint64_t* Uptr,
                const uint64_t* Vptr, int64_t b0, int64_t b1, const int64_t* lr_ptr,
                const int2* lr_ent, const int64_t* tile_row0, const int32_t* tile_m,
                int64_t n_tiles, const void* xm, void* t, int kcap, double* yacc, cudaStream_t s)
{
    const int64_t nb = b1 - b0;
    if (nb <= 0) return;
    if (precision == HM_PREC_FP64) {
        k_np_vtx<double><<<grid_for(nb * 32), NT, 0, s>>>(ablk, rank, Vptr, b0, nb,
                                                          static_cast<const double*>(xm),
                                                          static_cast<double*>(t), kcap);
        note_launch();
        if (n_tiles > 0)
            k_np_apply<double><<<grid_for(n_tiles * 32), NT, 0, s>>>(
                lr_ptr, lr_ent, ablk, rank, Uptr, tile_row0, tile_m, n_tiles, b0, b1,
                static_cast<const double*>(t), kcap, yacc);
    } else {
        k_np_vtx<float><<<grid_for(nb * 32), NT, 0, s>>>(ablk, rank, Vptr, b0, nb,
                                                         static_cast<const float*>(xm),
                                                         static_cast<float*>(t), kcap);
        note_launch();
        if (n_tiles > 0)
            k_np_apply<float><<<grid_for(n_tiles * 32), NT, 0, s>>>(
                lr_ptr, lr_ent, ablk, rank, Uptr, tile_row0, tile_m, n_tiles, b0, b1,
                static_cast<const float*>(t), kcap, yacc);
    }
    if (n_tiles > 0) note_launch();
    HM_LAUNCH("np low-rank part");
}

void np_near(int precision, const KernelParams& kp, const DeviceCoords& X, const Blk* dblk,
             const int64_t* dn_ptr, const int2* dn_ent, const int64_t* tile_row0,
             const int32_t* tile_m, int64_t n_tiles, const void* xm, double* yacc, cudaStream_t s)
{
    if (n_tiles <= 0) return;
    const unsigned g = grid_for(n_tiles * 32);
    if (precision == HM_PREC_FP64) {
        const double* xd = static_cast<const double*>(xm);
        if (kp.kernel == HM_GAUSSIAN)
            k_np_near<double, HM_GAUSSIAN><<<g, NT, 0, s>>>(kp, X, dblk, dn_ptr, dn_ent, tile_row0,
                                                            tile_m, n_tiles, xd, yacc);
        else
            k_np_near<double, HM_MATERN32><<<g, NT, 0, s>>>(kp, X, dblk, dn_ptr, dn_ent, tile_row0,
                                                            tile_m, n_tiles, xd, yacc);
    } else {
        const float* xf = static_cast<const float*>(xm);
        if (kp.kernel == HM_GAUSSIAN)
            k_np_near<float, HM_GAUSSIAN><<<g, NT, 0, s>>>(kp, X, dblk, dn_ptr, dn_ent, tile_row0,
                                                           tile_m, n_tiles, xf, yacc);
        else
            k_np_near<float, HM_MATERN32><<<g, NT, 0, s>>>(kp, X, dblk, dn_ptr, dn_ent, tile_row0,
                                                           tile_m, n_tiles, xf, yacc);
    }
    note_launch();
    HM_LAUNCH("np near field");
}

void np_finish(const int64_t* perm, const double* sig_row, double sigma2, int64_t N,
               const double* yacc, const double* x, double* y, int accumulate, cudaStream_t s)
{
    if (N <= 0) return;
    k_np_finish<<<grid_for(N), NT, 0, s>>>(perm, sig_row, sigma2, N, yacc, x, y, accumulate);
    note_launch();
    HM_LAUNCH("np finish");
}

}  // namespace hm
