// hm_mvp.cu -- batched H-matrix-vector product (Alg. 3 in the batched form
// of Sec. 5.4): x is permuted into Morton order (Sec. 5.1), t_b = V_b^T x|sigma
// is formed for every admissible leaf, and each row tile (a leaf cluster of the
// cluster tree) gathers, in a fixed order, U_b(rows, :) t_b of every
// admissible leaf whose tau contains it and A_b(rows, :) x|sigma of every
// dense leaf whose tau contains it. The gather replaces a scatter-add with
// atomics, so the result is deterministic; the last step adds sigma^2 x and
// writes y in the caller's order.
//
// Traffic per product: every factor entry and every near-field entry is read
// exactly once; x is gathered once (L2-resident reuse), y written once.
#include "hm_kernel_fn.cuh"

namespace hm {

namespace {

constexpr int NT = 256;
constexpr int VT_NT = 256;        // threads per CTA of the V^T x kernel
constexpr int VCH = 256;          // columns per V^T x work item (8 per lane)
constexpr int TILE_NT = 128;      // threads per CTA of the gather kernel
constexpr int TILE_WARPS = TILE_NT / 32;
constexpr int TROWS = 64;         // rows handled per pass of a tile

inline unsigned grid_for(int64_t n, int nt = NT) { return (unsigned)ceil_div(n, nt); }

int bits_for(int64_t n)
{
    int b = 0;
    while ((1ll << b) < n) ++b;
    return b;
}

// ------------------------------------------------------------------ product
template <class R>
__global__ void k_gather_x(const double* __restrict__ x, const int64_t* __restrict__ perm,
                           int64_t N, R* __restrict__ xm)
{
    int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i < N) xm[i] = (R)x[perm[i]];
}

// t partials: one warp per (block, 256-column chunk); lane j holds x of 8
// columns and each factor column is reduced with shuffles.
template <class R>
__global__ void __launch_bounds__(VT_NT)
k_vtx(const Blk* __restrict__ blk, const int32_t* __restrict__ rank,
      const uint64_t* __restrict__ Vptr, const int2* __restrict__ items, int64_t nitems,
      const int64_t* __restrict__ dst, const R* __restrict__ xm, R* __restrict__ t,
      R* __restrict__ tp)
{
    const int64_t w = ((int64_t)blockIdx.x * VT_NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nitems) return;
    const int2 it = items[w];
    const int b = it.x, c0 = it.y;
    const Blk B = blk[b];
    const int k = rank[b];
    const int n = B.n;
    const int cn = min(VCH, n - c0);
    const R* __restrict__ V = reinterpret_cast<const R*>(Vptr[b]);
    R xs[VCH / 32];
#pragma unroll
    for (int q = 0; q < VCH / 32; ++q) {
        const int jj = lane + 32 * q;
        xs[q] = (jj < cn) ? xm[B.col0 + c0 + jj] : R(0);
    }
    const int64_t d = dst[w];
    R* out = d >= 0 ? tp + d : t + (-d - 1);
    for (int l = 0; l < k; ++l) {
        const R* Vl = V + (int64_t)l * n + c0;
        R s = 0;
#pragma unroll
        for (int q = 0; q < VCH / 32; ++q) {
            const int jj = lane + 32 * q;
            if (jj < cn) s += Vl[jj] * xs[q];
        }
        s = warp_sum(s);
        if (lane == 0) out[l] = s;
    }
}

// Sum the partials of blocks that span several column chunks (fixed order).
template <class R>
__global__ void k_tsum(const int32_t* __restrict__ multi, int64_t nmulti,
                       const int32_t* __restrict__ rank, const int32_t* __restrict__ first,
                       const int32_t* __restrict__ count, const int64_t* __restrict__ dst,
                       const int64_t* __restrict__ toff, const R* __restrict__ tp,
                       R* __restrict__ t)
{
    const int64_t q = (int64_t)blockIdx.x;
    if (q >= nmulti) return;
    const int b = multi[q];
    const int k = rank[b];
    for (int l = threadIdx.x; l < k; l += blockDim.x) {
        R s = 0;
        for (int c = 0; c < count[b]; ++c) s += tp[dst[first[b] + c] + l];
        t[toff[b] + l] = s;
    }
}

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

template <class R, int FMT>
__device__ __forceinline__ R near_at(const void* store, int64_t o, int64_t mn, int64_t e)
{
    if (FMT == HM_NEAR_FP64) return (R) static_cast<const double*>(store)[o + e];
    if (FMT == HM_NEAR_FP32) return (R) static_cast<const float*>(store)[o + e];
    if (FMT == HM_NEAR_BF16X2) {
        const __nv_bfloat16* S = static_cast<const __nv_bfloat16*>(store) + 2 * o;
        return (R)(__bfloat162float(S[e]) + __bfloat162float(S[mn + e]));
    }
    return (R)__bfloat162float(static_cast<const __nv_bfloat16*>(store)[o + e]);
}

// One CTA per row tile; warps take the tile's gather entries round-robin and
// lanes own rows lane and lane + 32 of the current 64-row pass.
template <class R, int FMT>
__global__ void __launch_bounds__(TILE_NT)
k_tile(MvpPlan P, const R* __restrict__ xm, const R* __restrict__ t, const double* __restrict__ x,
       double* __restrict__ y, int accumulate)
{
    __shared__ double part[TILE_WARPS][TROWS];
    const int64_t tile = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t r0 = P.tile_row0[tile];
    const int mt = P.tile_m[tile];
    const int64_t l0 = P.lr_ptr[tile], l1 = P.lr_ptr[tile + 1];
    const int64_t d0 = P.dn_ptr[tile], d1 = P.dn_ptr[tile + 1];
    for (int rp = 0; rp < mt; rp += TROWS) {
        const int rows = min(TROWS, mt - rp);
        Acc<R> acc0, acc1;
        const int i0 = lane, i1 = lane + 32;
        // low-rank contributions U_b(rows, :) t_b
        for (int64_t e = l0 + w; e < l1; e += TILE_WARPS) {
            const int2 en = P.lr_ent[e];
            const int b = en.x;
            const int k = P.rank[b];
            const int m = P.ablk[b].m;
            const R* __restrict__ U = reinterpret_cast<const R*>(P.Uptr[b]) + en.y + rp;
            const R* __restrict__ tb = t + P.toff[b];
            R s0 = 0, s1 = 0;
            for (int l = 0; l < k; ++l) {
                const R tl = tb[l];
                const R* Ul = U + (int64_t)l * m;
                if (i0 < rows) s0 += Ul[i0] * tl;
                if (i1 < rows) s1 += Ul[i1] * tl;
            }
            acc0.add(s0);
            acc1.add(s1);
        }
        // dense contributions A_b(rows, :) x|sigma
        for (int64_t e = d0 + w; e < d1; e += TILE_WARPS) {
            const int2 en = P.dn_ent[e];
            const int b = en.x;
            const Blk B = P.dblk[b];
            const int64_t o = P.doff[b];
            const int64_t mn = (int64_t)B.m * B.n;
            const R* __restrict__ xs = xm + B.col0;
            R s0 = 0, s1 = 0;
            const int ra = en.y + rp + i0, rb = en.y + rp + i1;
            for (int j = 0; j < B.n; ++j) {
                const R xj = xs[j];
                const int64_t cj = (int64_t)j * B.m;
                if (i0 < rows) s0 += near_at<R, FMT>(P.near, o, mn, cj + ra) * xj;
                if (i1 < rows) s1 += near_at<R, FMT>(P.near, o, mn, cj + rb) * xj;
            }
            acc0.add(s0);
            acc1.add(s1);
        }
        part[w][i0] = acc0.value();
        part[w][i1] = acc1.value();
        __syncthreads();
        if ((int)threadIdx.x < rows) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < TILE_WARPS; ++q) s += part[q][threadIdx.x];
            const int64_t row = r0 + rp + threadIdx.x;
            const int64_t dst = P.perm[row];
            const double sg = P.sig_row ? P.sig_row[row] : P.sigma2;
            const double v = s + sg * x[dst];
            y[dst] = accumulate ? y[dst] + v : v;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ lists
// Tile index of a row: last tile with tile_row0 <= row.
__device__ __forceinline__ int64_t tile_of(const int64_t* __restrict__ tr0, int64_t nt,
                                           int64_t row)
{
    int64_t lo = 0, hi = nt - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (tr0[mid] <= row) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_tile_span(const Blk* __restrict__ blk, int64_t nb,
                            const int64_t* __restrict__ tr0, int64_t nt,
                            int64_t* __restrict__ first, int64_t* __restrict__ cnt)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= nb) return;
    const Blk B = blk[b];
    int64_t f = tile_of(tr0, nt, B.row0);
    int64_t l = tile_of(tr0, nt, B.row0 + B.m - 1);
    first[b] = f;
    cnt[b] = l - f + 1;
}

__global__ void k_emit_entries(const Blk* __restrict__ blk, int64_t nb,
                               const int64_t* __restrict__ first,
                               const int64_t* __restrict__ cnt, const int64_t* __restrict__ off,
                               const int64_t* __restrict__ tr0, uint64_t* __restrict__ key,
                               uint32_t* __restrict__ val, int2* __restrict__ ent,
                               int32_t* __restrict__ tcount)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= nb) return;
    const Blk B = blk[b];
    for (int64_t q = 0; q < cnt[b]; ++q) {
        int64_t e = off[b] + q, tl = first[b] + q;
        key[e] = (uint64_t)tl;
        val[e] = (uint32_t)e;
        ent[e] = make_int2((int)b, (int)(tr0[tl] - B.row0));
        atomicAdd(&tcount[tl], 1);
    }
}

__global__ void k_gather_ent(const int2* __restrict__ in, const uint32_t* __restrict__ idx,
                             int64_t n, int2* __restrict__ out)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e < n) out[e] = in[idx[e]];
}

__global__ void k_i32_to_i64(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ out)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e < n) out[e] = in[e];
}

// Build one CSR over tiles for a list of blocks.
void build_csr(const Blk* blk, int64_t nb, const int64_t* tr0, int64_t nt,
               DevBuf<int64_t>& ptr, DevBuf<int2>& ent, cudaStream_t s)
{
    ptr.alloc(nt + 1, s);
    DevBuf<int32_t> tcount(nt + 1, s);
    HM_CUDA(cudaMemsetAsync(tcount.p, 0, (nt + 1) * sizeof(int32_t), s));
    if (nb == 0) {
        HM_CUDA(cudaMemsetAsync(ptr.p, 0, (nt + 1) * sizeof(int64_t), s));
        ent.alloc(1, s);
        return;
    }
    DevBuf<int64_t> first(nb, s), cnt(nb, s), off(nb, s), tot(1, s);
    k_tile_span<<<grid_for(nb), NT, 0, s>>>(blk, nb, tr0, nt, first.p, cnt.p); note_launch();
    scan_exclusive_i64(cnt.p, off.p, nb, tot.p, s);
    int64_t E = 0;
    HM_CUDA(cudaMemcpyAsync(&E, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    if (E > (int64_t)UINT32_MAX) fail(HM_EOVERFLOW, "too many gather entries");
    DevBuf<uint64_t> key(E, s);
    DevBuf<uint32_t> val(E, s);
    DevBuf<int2> tmp(E, s);
    k_emit_entries<<<grid_for(nb), NT, 0, s>>>(blk, nb, first.p, cnt.p, off.p, tr0, key.p,
                                               val.p, tmp.p, tcount.p); note_launch();
    HM_LAUNCH("emit entries");
    radix_sort_u64_u32(key.p, val.p, E, bits_for(nt + 1), s);
    ent.alloc(E, s);
    k_gather_ent<<<grid_for(E), NT, 0, s>>>(tmp.p, val.p, E, ent.p); note_launch();
    DevBuf<int64_t> c64(nt + 1, s);
    k_i32_to_i64<<<grid_for(nt + 1), NT, 0, s>>>(tcount.p, nt + 1, c64.p); note_launch();
    scan_exclusive_i64(c64.p, ptr.p, nt + 1, nullptr, s);
    HM_LAUNCH("csr");
}

__global__ void k_vitems_count(const Blk* __restrict__ blk, const int32_t* __restrict__ rank,
                               int64_t nb, int64_t* __restrict__ cnt,
                               int64_t* __restrict__ multi_t, int32_t* __restrict__ ismulti,
                               int64_t* __restrict__ rk)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= nb) return;
    int k = rank[b];
    int64_t c = k > 0 ? ceil_div(blk[b].n, VCH) : 0;
    cnt[b] = c;
    multi_t[b] = c > 1 ? c * k : 0;
    ismulti[b] = c > 1 ? 1 : 0;
    rk[b] = k;
}

__global__ void k_vitems_emit(const Blk* __restrict__ blk, int64_t nb,
                              const int64_t* __restrict__ cnt, const int64_t* __restrict__ ioff,
                              const int64_t* __restrict__ poff, const int64_t* __restrict__ toff,
                              const int32_t* __restrict__ rank, const int32_t* __restrict__ moff,
                              int2* __restrict__ items, int64_t* __restrict__ dst,
                              int32_t* __restrict__ first, int32_t* __restrict__ count,
                              int32_t* __restrict__ multi)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= nb) return;
    int64_t c = cnt[b];
    first[b] = (int32_t)ioff[b];
    count[b] = (int32_t)c;
    for (int64_t q = 0; q < c; ++q) {
        items[ioff[b] + q] = make_int2((int)b, (int)(q * VCH));
        dst[ioff[b] + q] = (c > 1) ? poff[b] + q * rank[b] : -(toff[b] + 1);
    }
    if (c > 1) multi[moff[b]] = (int32_t)b;
}

}  // namespace

void mvp_build_lists(const Blk* ablk, const int32_t* rank, int64_t n_adm, const Blk* dblk,
                     int64_t n_dense, const int64_t* leaf_row0, const int32_t* leaf_m,
                     int64_t n_tiles, MvpLists& L, cudaStream_t s)
{
    L.n_tiles = n_tiles;
    build_csr(ablk, n_adm, leaf_row0, n_tiles, L.lr_ptr, L.lr_ent, s);
    build_csr(dblk, n_dense, leaf_row0, n_tiles, L.dn_ptr, L.dn_ent, s);
    // t offsets and V^T x work items
    const int64_t nb = std::max<int64_t>(n_adm, 1);
    DevBuf<int64_t> cnt(nb, s), ioff(nb, s), mt(nb, s), poff(nb, s), rk(nb, s), tot(3, s);
    DevBuf<int32_t> ism(nb, s), moff(nb, s);
    L.toff.alloc(nb, s);
    L.tsum_first.alloc(nb, s);
    L.tsum_count.alloc(nb, s);
    int64_t h[3] = {0, 0, 0};
    int32_t hm = 0;
    if (n_adm > 0) {
        k_vitems_count<<<grid_for(n_adm), NT, 0, s>>>(ablk, rank, n_adm, cnt.p, mt.p, ism.p, rk.p); note_launch();
        scan_exclusive_i64(cnt.p, ioff.p, n_adm, tot.p, s);
        scan_exclusive_i64(mt.p, poff.p, n_adm, tot.p + 1, s);
        scan_exclusive_i64(rk.p, L.toff.p, n_adm, tot.p + 2, s);
        DevBuf<int32_t> mtot(1, s);
        scan_exclusive_i32(ism.p, moff.p, n_adm, mtot.p, s);
        HM_CUDA(cudaMemcpyAsync(h, tot.p, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(&hm, mtot.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
    }
    L.n_vitems = h[0];
    L.tpart_len = h[1];
    L.t_len = h[2];
    L.n_multi = hm;
    L.vitems.alloc(std::max<int64_t>(L.n_vitems, 1), s);
    L.tpart_off.alloc(std::max<int64_t>(L.n_vitems, 1), s);
    L.multi.alloc(std::max<int64_t>(L.n_multi, 1), s);
    if (n_adm > 0)
        k_vitems_emit<<<grid_for(n_adm), NT, 0, s>>>(ablk, n_adm, cnt.p, ioff.p, poff.p,
                                                     L.toff.p, rank, moff.p, L.vitems.p,
                                                     L.tpart_off.p, L.tsum_first.p,
                                                     L.tsum_count.p, L.multi.p); note_launch();
    HM_LAUNCH("vitems");
}

void mvp_alloc_work(const MvpPlan& P, MvpWork& W, cudaStream_t s)
{
    if (P.precision == HM_PREC_FP64) {
        W.xm64.alloc(std::max<int64_t>(P.Ntot, 1), s);
        W.t64.alloc(std::max<int64_t>(P.t_len, 1), s);
        W.tp64.alloc(std::max<int64_t>(P.tpart_len, 1), s);
    } else {
        W.xm32.alloc(std::max<int64_t>(P.Ntot, 1), s);
        W.t32.alloc(std::max<int64_t>(P.t_len, 1), s);
        W.tp32.alloc(std::max<int64_t>(P.tpart_len, 1), s);
    }
}

namespace {

template <class R, int FMT>
void run_typed(const MvpPlan& P, R* xm, R* t, R* tp, const double* x, double* y,
               int accumulate, cudaStream_t s, MvpTimer* timer)
{
    MvpTimer::Rec* rec = timer ? timer->begin() : nullptr;
    if (rec) HM_CUDA(cudaEventRecord(rec->e[0], s));
    k_gather_x<R><<<grid_for(P.Ntot), NT, 0, s>>>(x, P.perm, P.Ntot, xm); note_launch();
    if (rec) HM_CUDA(cudaEventRecord(rec->e[1], s));
    if (P.n_vitems > 0)
        k_vtx<R><<<grid_for(P.n_vitems * 32, VT_NT), VT_NT, 0, s>>>(
            P.ablk, P.rank, P.Vptr, P.vitems, P.n_vitems, P.tpart_off, xm, t, tp); note_launch();
    if (P.n_multi > 0)
        k_tsum<R><<<(unsigned)P.n_multi, 64, 0, s>>>(P.multi, P.n_multi, P.rank, P.tsum_first,
                                                     P.tsum_count, P.tpart_off, P.toff, tp, t); note_launch();
    if (rec) HM_CUDA(cudaEventRecord(rec->e[2], s));
    if (P.n_tiles > 0)
        k_tile<R, FMT><<<(unsigned)P.n_tiles, TILE_NT, 0, s>>>(P, xm, t, x, y, accumulate); note_launch();
    if (rec) HM_CUDA(cudaEventRecord(rec->e[3], s));
    HM_LAUNCH("matvec");
}

}  // namespace

MvpTimer::Rec* MvpTimer::begin()
{
    Rec r;
    if (!pool.empty()) {
        r = pool.back();
        pool.pop_back();
    } else {
        for (int k = 0; k < 4; ++k) HM_CUDA(cudaEventCreate(&r.e[k]));
    }
    recs.push_back(r);
    return &recs.back();
}

void MvpTimer::collect()
{
    for (Rec& r : recs) {
        HM_CUDA(cudaEventSynchronize(r.e[3]));
        float a = 0, b = 0, c = 0;
        HM_CUDA(cudaEventElapsedTime(&a, r.e[0], r.e[1]));
        HM_CUDA(cudaEventElapsedTime(&b, r.e[1], r.e[2]));
        HM_CUDA(cudaEventElapsedTime(&c, r.e[2], r.e[3]));
        t_gather += a;
        t_vtx += b;
        t_tile += c;
        t_total += a + b + c;
        ++count;
        pool.push_back(r);
    }
    recs.clear();
}

MvpTimer::~MvpTimer()
{
    for (Rec& r : recs) pool.push_back(r);
    for (Rec& r : pool)
        for (int k = 0; k < 4; ++k) cudaEventDestroy(r.e[k]);
}

namespace {

}  // namespace

void mvp_run(const MvpPlan& P, MvpWork& W, const double* x, double* y, int accumulate,
             cudaStream_t s, MvpTimer* timer)
{
    if (P.precision == HM_PREC_FP64) {
        run_typed<double, HM_NEAR_FP64>(P, W.xm64.p, W.t64.p, W.tp64.p, x, y, accumulate, s, timer);
        return;
    }
    switch (P.near_format) {
    case HM_NEAR_FP64:
        run_typed<float, HM_NEAR_FP64>(P, W.xm32.p, W.t32.p, W.tp32.p, x, y, accumulate, s, timer);
        break;
    case HM_NEAR_FP32:
        run_typed<float, HM_NEAR_FP32>(P, W.xm32.p, W.t32.p, W.tp32.p, x, y, accumulate, s, timer);
        break;
    case HM_NEAR_BF16X2:
        run_typed<float, HM_NEAR_BF16X2>(P, W.xm32.p, W.t32.p, W.tp32.p, x, y, accumulate, s, timer);
        break;
    default:
        run_typed<float, HM_NEAR_BF16>(P, W.xm32.p, W.t32.p, W.tp32.p, x, y, accumulate, s, timer);
        break;
    }
}

}  // namespace hm
