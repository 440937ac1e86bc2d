// hm_np.cu -- kernels of the product that stores nothing but the block
// structure (the paper's non-precomputed mode, Sec. 5.4 with the factors and
// the dense blocks recomputed for every product): per pass of admissible
// leaves the ACA factors are rebuilt in a bounded scratch area and applied at
// once, and the dense leaves are evaluated inside the product.
//
// Determinism: every row of y is one running sum in double, fed in a fixed
// order: the admissible leaves of the row's tile in block order (the passes
// take consecutive block ranges), then the near-field item sums of the tile
// in item order, each summed in a fixed pattern of warps and columns. In
// symmetric mode a pass applies its canonical leaves and their mirror leaves,
// which lie later in block order, so a row's leaves enter in (pass, block)
// order: fixed for a given scratch size, equal to rounding across sizes.
#include "hm_kernel_fn.cuh"
#include "hm_stream.cuh"

#include <vector>

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

// Work lists, built once: V^T x items (block, first column) of VCH columns,
// every block's items consecutive from vptr[b]; apply items (tile, first
// entry, end entry) of at most NP_AE entries of the tile's list of
// admissible leaves, every tile's items consecutive from aptr[tile].
constexpr int NP_AE = 16;

__global__ void k_np_vcount(const Blk* __restrict__ blk, int64_t n, int64_t* __restrict__ cnt)
{
    const int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b < n) cnt[b] = ceil_div((int64_t)blk[b].n, (int64_t)VCH);
}

__global__ void k_np_vemit(const Blk* __restrict__ blk, int64_t n, const int64_t* __restrict__ vptr,
                           int2* __restrict__ items)
{
    const int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    const int64_t c = vptr[b + 1] - vptr[b];
    for (int64_t q = 0; q < c; ++q) items[vptr[b] + q] = make_int2((int)b, (int)(q * VCH));
}

__global__ void k_np_acount(const int64_t* __restrict__ lr_ptr, int64_t nt, int64_t* __restrict__ cnt)
{
    const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q < nt) cnt[q] = ceil_div(lr_ptr[q + 1] - lr_ptr[q], (int64_t)NP_AE);
}

__global__ void k_np_aemit(const int64_t* __restrict__ lr_ptr, int64_t nt,
                           const int64_t* __restrict__ aptr, int3* __restrict__ items)
{
    const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= nt) return;
    const int64_t e0 = lr_ptr[q], e1 = lr_ptr[q + 1];
    for (int64_t a = aptr[q]; a < aptr[q + 1]; ++a) {
        const int64_t f = e0 + (a - aptr[q]) * NP_AE;
        items[a] = make_int3((int)q, (int)f, (int)min(e1, f + NP_AE));
    }
}

// t partials of the V^T x items vi0 .. vi0 + ni - 1: one warp per item, lane
// j sums the columns j, j + 32, ... of the item's chunk for every factor row
// l, the lane sums meet in the xor butterfly; partial (item, l) goes to
// tp[(item - vi0) kcap + l].
// With pidx (symmetric handles) the pass's items are items[pidx[vi0 + w]].
template <class R>
__global__ void k_np_vtx(const Blk* __restrict__ blk, const int32_t* __restrict__ rank,
                         const uint64_t* __restrict__ Vptr, const int2* __restrict__ items,
                         const int64_t* __restrict__ pidx, int64_t vi0, int64_t ni,
                         const R* __restrict__ xm, R* __restrict__ tp, int kcap)
{
    const int64_t w = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= ni) return;
    const int2 it = items[pidx ? pidx[vi0 + w] : vi0 + w];
    const Blk B = blk[it.x];
    const int k = rank[it.x];
    const int n = B.n, c0 = it.y;
    const int cn = min(VCH, n - c0);
    const R* __restrict__ V = reinterpret_cast<const R*>(Vptr[it.x]) + c0;
    R xs[VCH / 32];
#pragma unroll
    for (int q = 0; q < VCH / 32; ++q) {
        const int jj = lane + 32 * q;
        xs[q] = jj < cn ? xm[B.col0 + c0 + jj] : R(0);
    }
    R* out = tp + w * kcap;
    for (int l = 0; l < k; ++l) {
        const R* Vl = V + (int64_t)l * n;
        R s = R(0);
#pragma unroll
        for (int q = 0; q < VCH / 32; ++q) {
            const int jj = lane + 32 * q;
            if (jj < cn) s = fma(__ldcs(Vl + jj), xs[q], s);
        }
        s = warp_sum(s);
        if (lane == 0) out[l] = s;
    }
}

// t_b = sum of its items' partials in item order, for the blocks b0 .. b0 +
// nb - 1 (one warp per block); t_b starts at t + (b - b0) kcap. With pblk
// (symmetric handles) the blocks are pblk[b0 + w] and the first partial of
// block b is pfirst[b].
template <class R>
__global__ void k_np_tsum(const int64_t* __restrict__ vptr, const int64_t* __restrict__ pblk,
                          const int64_t* __restrict__ pfirst, int64_t b0, int64_t nb,
                          const int32_t* __restrict__ rank, int64_t vi0, const R* __restrict__ tp,
                          R* __restrict__ t, int kcap)
{
    const int64_t w = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nb) return;
    const int64_t b = pblk ? pblk[b0 + w] : b0 + w;
    const int k = rank[b];
    const int64_t f = pblk ? pfirst[b] : vptr[b] - vi0, c = vptr[b + 1] - vptr[b];
    for (int l = lane; l < k; l += 32) {
        R s = R(0);
        for (int64_t q = 0; q < c; ++q) s += tp[(f + q) * kcap + l];
        t[w * kcap + l] = s;
    }
}

// U_b t_b over the admissible leaves b0 <= b < b1 of every apply item, added
// to the item's running row sums in entry (= block) order; one warp per item,
// lane i takes rows i, i + 32, ... (item_acc holds ld sums per item).
template <class R>
__global__ void k_np_apply(const int3* __restrict__ items, int64_t n_items,
                           const int2* __restrict__ lr_ent, const Blk* __restrict__ blk,
                           const int32_t* __restrict__ rank, const uint64_t* __restrict__ Uptr,
                           const int32_t* __restrict__ tile_m, int64_t b0, int64_t b1,
                           const R* __restrict__ t, int kcap, int ld, double* __restrict__ item_acc)
{
    const int64_t w = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_items) return;
    const int3 it = items[w];
    int e0 = it.y, e1 = it.z;
    // the item's entries in this pass (entries ascend by block)
    while (e0 < e1 && lr_ent[e0].x < b0) ++e0;
    if (e0 >= e1 || lr_ent[e0].x >= b1) return;
    const int mt = tile_m[it.x];
    for (int i = lane; i < mt; i += 32) {
        double v = item_acc[w * ld + i];
        for (int e = e0; e < e1; ++e) {
            const int2 en = lr_ent[e];
            if (en.x >= b1) break;
            const int k = rank[en.x];
            const int m = blk[en.x].m;
            const R* __restrict__ U = reinterpret_cast<const R*>(Uptr[en.x]) + en.y + i;
            const R* __restrict__ tb = t + (int64_t)(en.x - b0) * kcap;
            R c = R(0);
            for (int l = 0; l < k; ++l) c = fma(U[(int64_t)l * m], tb[l], c);
            v += (double)c;
        }
        item_acc[w * ld + i] = v;
    }
}

// Symmetric handles: U_b t_b over the entries of every apply item whose leaf
// is in pass q (canonical leaves of the pass and their mirror leaves, whose
// U is the partner's V), in entry order; t_b at t + tidx[b] kcap.
template <class R>
__global__ void k_np_apply_sym(const int3* __restrict__ items, int64_t n_items,
                               const int2* __restrict__ lr_ent, const Blk* __restrict__ blk,
                               const int32_t* __restrict__ rank, const uint64_t* __restrict__ Uptr,
                               const int32_t* __restrict__ tile_m, const int32_t* __restrict__ passid,
                               const int32_t* __restrict__ tidx, int q, const R* __restrict__ t,
                               int kcap, int ld, double* __restrict__ item_acc)
{
    const int64_t w = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_items) return;
    const int3 it = items[w];
    bool any = false;
    for (int e = it.y; e < it.z; ++e) any |= passid[lr_ent[e].x] == q;
    if (!any) return;
    const int mt = tile_m[it.x];
    for (int i = lane; i < mt; i += 32) {
        double v = item_acc[w * ld + i];
        for (int e = it.y; e < it.z; ++e) {
            const int2 en = lr_ent[e];
            if (passid[en.x] != q) continue;
            const int k = rank[en.x];
            const int m = blk[en.x].m;
            const R* __restrict__ U = reinterpret_cast<const R*>(Uptr[en.x]) + en.y + i;
            const R* __restrict__ tb = t + (int64_t)tidx[en.x] * kcap;
            R c = R(0);
            for (int l = 0; l < k; ++l) c = fma(U[(int64_t)l * m], tb[l], c);
            v += (double)c;
        }
        item_acc[w * ld + i] = v;
    }
}

// y_m += the apply items' row sums of every tile, in item order (one warp per tile).
__global__ void k_np_apply_finish(const int64_t* __restrict__ aptr,
                                  const int64_t* __restrict__ tile_row0,
                                  const int32_t* __restrict__ tile_m, int64_t n_tiles, int ld,
                                  const double* __restrict__ item_acc, double* __restrict__ yacc)
{
    const int64_t tile = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= n_tiles) return;
    const int64_t r0 = tile_row0[tile];
    const int mt = tile_m[tile];
    const int64_t a0 = aptr[tile], a1 = aptr[tile + 1];
    for (int i = lane; i < mt; i += 32) {
        double sum = 0.0;
        for (int64_t q = a0; q < a1; ++q) sum += item_acc[q * ld + i];
        yacc[r0 + i] += sum;
    }
}

// The dense leaves of the product, entries phi(y_i, y_j) evaluated on the fly
// (the same kernel functions as the stored near field). One CTA per work item
// of the gather (a run of at most 4096 columns of one row tile's near-field
// column stream, column c the point ncol_x[c]): warp w takes the columns w,
// w + 8, ... of the item, lane i the rows i and i + 32 of each 64-row window;
// plain sums over 16 of a warp's columns enter a compensated sum (double sum
// in FP64), the warps' sums add in warp order into the item's partial row
// sums, and k_np_near_finish adds the items of a tile in item order.
constexpr int NN_W = 8;
constexpr int NN_ROWS = 64;

// A point held by lane src, to every lane of the warp.
__device__ __forceinline__ Pt<double> shfl_pt(const Pt<double>& p, int src)
{
    Pt<double> o;
#pragma unroll
    for (int i = 0; i < 3; ++i) o.x[i] = __shfl_sync(0xffffffffu, p.x[i], src);
    return o;
}

__device__ __forceinline__ Pt<float> shfl_pt(const Pt<float>& p, int src)
{
    Pt<float> o;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o.h[i] = __shfl_sync(0xffffffffu, p.h[i], src);
        o.l[i] = __shfl_sync(0xffffffffu, p.l[i], src);
    }
    return o;
}

template <class R, int KERN>
__global__ void __launch_bounds__(NN_W * 32)
k_np_near(KernelParams kp, DeviceCoords X, const int3* __restrict__ items,
          const int64_t* __restrict__ ucol_ptr, const int64_t* __restrict__ ncol_ptr,
          const int32_t* __restrict__ ncol_x, const int64_t* __restrict__ tile_row0,
          const int32_t* __restrict__ tile_m, int max_ld, const R* __restrict__ xm,
          double* __restrict__ part)
{
    __shared__ double ps[NN_W][NN_ROWS];
    const int64_t item = blockIdx.x;
    const int3 it = items[item];
    const int64_t tile = it.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = tile_row0[tile];
    const int mt = tile_m[tile];
    const int64_t nu = ucol_ptr[tile + 1] - ucol_ptr[tile];
    const int64_t nc0 = ncol_ptr[tile];
    const int64_t cb = it.y > nu ? it.y - nu : 0, ce = it.z > nu ? it.z - nu : 0;
    const R c = kconst<R>(kp);
    for (int rw = 0; rw < mt; rw += NN_ROWS) {
        const int ia = rw + lane, ib = rw + lane + 32;
        const Pt<R> pa = load_pt<R>(X, r0 + min(ia, mt - 1));
        const Pt<R> pb = load_pt<R>(X, r0 + min(ib, mt - 1));
        Acc<R> aa, ab;
        R sa = R(0), sb = R(0);
        int cnt = 0;
        // the warp's columns w, w + NN_W, ... in batches of 32: lane L fetches
        // column base + NN_W L (index, point, x) for the whole batch at once,
        // then the batch is walked in column order with the column's point
        // and x taken from its lane
        for (int64_t base = cb + w; base < ce; base += (int64_t)NN_W * 32) {
            const int64_t mycol = base + (int64_t)NN_W * lane;
            Pt<R> pl = load_pt<R>(X, r0);          // any valid point for idle lanes
            R xl = R(0);
            if (mycol < ce) {
                const int32_t q = ncol_x[nc0 + mycol];
                pl = load_pt<R>(X, q);
                xl = xm[q];
            }
            const int nt = (int)min((int64_t)32, (ce - base + NN_W - 1) / NN_W);
            for (int t = 0; t < nt; ++t) {
                const Pt<R> pq = shfl_pt(pl, t);
                const R xq = __shfl_sync(0xffffffffu, xl, t);
                sa = fma(phi<KERN>(dist2(pa, pq), c), xq, sa);
                sb = fma(phi<KERN>(dist2(pb, pq), c), xq, sb);
                if (++cnt == 16) {
                    aa.add(sa);
                    ab.add(sb);
                    sa = sb = R(0);
                    cnt = 0;
                }
            }
        }
        aa.add(sa);
        ab.add(sb);
        ps[w][lane] = aa.value();
        ps[w][lane + 32] = ab.value();
        __syncthreads();
        const int rows = min(NN_ROWS, mt - rw);
        if ((int)threadIdx.x < rows) {
            double sum = 0.0;
#pragma unroll
            for (int q = 0; q < NN_W; ++q) sum += ps[q][threadIdx.x];
            part[item * max_ld + rw + threadIdx.x] = sum;
        }
        __syncthreads();
    }
}

// y_m += the near-field item sums of every tile, in item order (one warp per tile).
__global__ void k_np_near_finish(const int64_t* __restrict__ item_ptr,
                                 const int64_t* __restrict__ tile_row0,
                                 const int32_t* __restrict__ tile_m, int64_t n_tiles, int max_ld,
                                 const double* __restrict__ part, double* __restrict__ yacc)
{
    const int64_t tile = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= n_tiles) return;
    const int64_t r0 = tile_row0[tile];
    const int mt = tile_m[tile];
    const int64_t i0 = item_ptr[tile], i1 = item_ptr[tile + 1];
    for (int i = lane; i < mt; i += 32) {
        double sum = 0.0;
        for (int64_t q = i0; q < i1; ++q) sum += part[q * max_ld + i];
        yacc[r0 + i] += sum;
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

template <class R>
void launch_np_near(const KernelParams& kp, const DeviceCoords& X, unsigned g, const int3* items,
                    const int64_t* ucol_ptr, const int64_t* ncol_ptr, const int32_t* ncol_x,
                    const int64_t* tile_row0, const int32_t* tile_m, int max_ld, const R* xm,
                    double* part, cudaStream_t s)
{
    const int bs = NN_W * 32;
    if (kp.kernel == HM_GAUSSIAN)
        k_np_near<R, HM_GAUSSIAN><<<g, bs, 0, s>>>(kp, X, items, ucol_ptr, ncol_ptr, ncol_x,
                                                   tile_row0, tile_m, max_ld, xm, part);
    else if (kp.kernel == HM_MATERN32)
        k_np_near<R, HM_MATERN32><<<g, bs, 0, s>>>(kp, X, items, ucol_ptr, ncol_ptr, ncol_x,
                                                   tile_row0, tile_m, max_ld, xm, part);
    else
        k_np_near<R, HM_MATERN_K1><<<g, bs, 0, s>>>(kp, X, items, ucol_ptr, ncol_ptr, ncol_x,
                                                    tile_row0, tile_m, max_ld, xm, part);
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

void np_lists(const Blk* ablk, int64_t n_adm, const int64_t* lr_ptr, int64_t n_tiles,
              DevBuf<int64_t>& vptr, DevBuf<int2>& vitems, DevBuf<int64_t>& aptr,
              DevBuf<int3>& aitems, std::vector<int64_t>& h_vptr, int64_t& n_aitems, cudaStream_t s)
{
    const int64_t nb = std::max<int64_t>(n_adm, 1);
    vptr.alloc(nb + 1, s);
    HM_CUDA(cudaMemsetAsync(vptr.p, 0, (nb + 1) * sizeof(int64_t), s));
    h_vptr.assign(n_adm + 1, 0);
    if (n_adm > 0) {
        DevBuf<int64_t> cnt(n_adm, s);
        k_np_vcount<<<grid_for(n_adm), NT, 0, s>>>(ablk, n_adm, cnt.p); note_launch();
        scan_exclusive_i64(cnt.p, vptr.p, n_adm, vptr.p + n_adm, s);
        HM_CUDA(cudaMemcpyAsync(h_vptr.data(), vptr.p, (n_adm + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
    }
    vitems.alloc(std::max<int64_t>(h_vptr[n_adm], 1), s);
    if (n_adm > 0) {
        k_np_vemit<<<grid_for(n_adm), NT, 0, s>>>(ablk, n_adm, vptr.p, vitems.p); note_launch();
    }
    aptr.alloc(n_tiles + 1, s);
    HM_CUDA(cudaMemsetAsync(aptr.p, 0, (n_tiles + 1) * sizeof(int64_t), s));
    n_aitems = 0;
    if (n_tiles > 0) {
        DevBuf<int64_t> cnt(n_tiles, s);
        k_np_acount<<<grid_for(n_tiles), NT, 0, s>>>(lr_ptr, n_tiles, cnt.p); note_launch();
        scan_exclusive_i64(cnt.p, aptr.p, n_tiles, aptr.p + n_tiles, s);
        HM_CUDA(cudaMemcpyAsync(&n_aitems, aptr.p + n_tiles, sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
    }
    aitems.alloc(std::max<int64_t>(n_aitems, 1), s);
    if (n_tiles > 0) {
        k_np_aemit<<<grid_for(n_tiles), NT, 0, s>>>(lr_ptr, n_tiles, aptr.p, aitems.p); note_launch();
    }
    HM_LAUNCH("np lists");
    HM_CUDA(cudaStreamSynchronize(s));
}

namespace {

template <class R>
void lowrank_typed(const Blk* ablk, const int32_t* rank, const uint64_t* Uptr,
                   const uint64_t* Vptr, int64_t b0, int64_t b1, const int64_t* vptr,
                   const int2* vitems, int64_t vi0, int64_t vi1, const int3* aitems,
                   int64_t n_aitems, const int2* lr_ent, const int32_t* tile_m, const R* x,
                   R* p, R* tt, int kcap, int ld, double* item_acc, const NpSymPass* sym,
                   cudaStream_t s)
{
    const int64_t nb = b1 - b0, ni = vi1 - vi0;
    if (ni > 0) {
        k_np_vtx<R><<<grid_for(ni * 32), NT, 0, s>>>(ablk, rank, Vptr, vitems,
                                                    sym ? sym->pitems : nullptr, vi0, ni, x, p,
                                                    kcap);
        note_launch();
    }
    k_np_tsum<R><<<grid_for(nb * 32), NT, 0, s>>>(vptr, sym ? sym->pblk : nullptr,
                                                  sym ? sym->pfirst : nullptr, b0, nb, rank, vi0,
                                                  p, tt, kcap);
    note_launch();
    if (n_aitems > 0) {
        if (sym)
            k_np_apply_sym<R><<<grid_for(n_aitems * 32), NT, 0, s>>>(
                aitems, n_aitems, lr_ent, ablk, rank, Uptr, tile_m, sym->passid, sym->tidx,
                sym->q, tt, kcap, ld, item_acc);
        else
            k_np_apply<R><<<grid_for(n_aitems * 32), NT, 0, s>>>(
                aitems, n_aitems, lr_ent, ablk, rank, Uptr, tile_m, b0, b1, tt, kcap, ld,
                item_acc);
        note_launch();
    }
}

}  // namespace

void np_lowrank(int precision, const Blk* ablk, const int32_t* rank, const uint64_t* Uptr,
                const uint64_t* Vptr, int64_t b0, int64_t b1, const int64_t* vptr,
                const int2* vitems, int64_t vi0, int64_t vi1, const int3* aitems,
                int64_t n_aitems, const int2* lr_ent, const int32_t* tile_m, const void* xm,
                void* tp, void* t, int kcap, int ld, double* item_acc, cudaStream_t s,
                const NpSymPass* sym)
{
    if (b1 - b0 <= 0) return;
    if (precision == HM_PREC_FP64)
        lowrank_typed<double>(ablk, rank, Uptr, Vptr, b0, b1, vptr, vitems, vi0, vi1, aitems,
                              n_aitems, lr_ent, tile_m, static_cast<const double*>(xm),
                              static_cast<double*>(tp), static_cast<double*>(t), kcap, ld,
                              item_acc, sym, s);
    else
        lowrank_typed<float>(ablk, rank, Uptr, Vptr, b0, b1, vptr, vitems, vi0, vi1, aitems,
                             n_aitems, lr_ent, tile_m, static_cast<const float*>(xm),
                             static_cast<float*>(tp), static_cast<float*>(t), kcap, ld,
                             item_acc, sym, s);
    HM_LAUNCH("np low-rank part");
}

void np_apply_finish(const int64_t* aptr, const int64_t* tile_row0, const int32_t* tile_m,
                     int64_t n_tiles, int ld, const double* item_acc, double* yacc, cudaStream_t s)
{
    if (n_tiles <= 0) return;
    k_np_apply_finish<<<grid_for(n_tiles * 32), NT, 0, s>>>(aptr, tile_row0, tile_m, n_tiles, ld,
                                                            item_acc, yacc);
    note_launch();
    HM_LAUNCH("np low-rank sums");
}

void np_near(int precision, const KernelParams& kp, const DeviceCoords& X, const int3* items,
             int64_t n_items, const int64_t* item_ptr, const int64_t* ucol_ptr,
             const int64_t* ncol_ptr, const int32_t* ncol_x, const int64_t* tile_row0,
             const int32_t* tile_m, int64_t n_tiles, int max_ld, const void* xm, double* part,
             double* yacc, cudaStream_t s)
{
    if (n_tiles <= 0 || n_items <= 0) return;
    if (n_items > 0x7fffffffll) fail(HM_EOVERFLOW, "too many near-field items for one launch");
    const unsigned g = (unsigned)n_items;
    if (precision == HM_PREC_FP64)
        launch_np_near<double>(kp, X, g, items, ucol_ptr, ncol_ptr, ncol_x, tile_row0, tile_m,
                               max_ld, static_cast<const double*>(xm), part, s);
    else
        launch_np_near<float>(kp, X, g, items, ucol_ptr, ncol_ptr, ncol_x, tile_row0, tile_m,
                              max_ld, static_cast<const float*>(xm), part, s);
    note_launch();
    k_np_near_finish<<<grid_for(n_tiles * 32), NT, 0, s>>>(item_ptr, tile_row0, tile_m, n_tiles,
                                                           max_ld, part, yacc);
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
