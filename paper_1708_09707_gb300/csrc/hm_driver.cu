// hm_driver.cu -- product driver, exports, conjugate gradients and the batched
// entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hm_handle.cuh"

namespace hm {

namespace {

constexpr int NT = 256;
inline unsigned grid_for(int64_t n) { return (unsigned)ceil_div(n, NT); }

__global__ void k_add_offset(int64_t* __restrict__ p, int64_t n, int64_t off)
{
    int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i < n) p[i] += off;
}

// Deterministic double dot product: a fixed grid of CTAs writes partial sums
// (fixed per-thread stride, fixed tree in the CTA), one CTA adds the partials
// in index order.
constexpr int DOT_BLOCKS = 1024;

__global__ void k_dot_part(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                           double* __restrict__ part)
{
    __shared__ double sm[NT];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)DOT_BLOCKS * NT)
        s += a[i] * b[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_dot_final(const double* __restrict__ part, double* __restrict__ out)
{
    __shared__ double sm[DOT_BLOCKS];
    for (int i = threadIdx.x; i < DOT_BLOCKS; i += blockDim.x) sm[i] = part[i];
    __syncthreads();
    for (int o = DOT_BLOCKS / 2; o > 0; o >>= 1) {
        for (int i = threadIdx.x; i < o; i += blockDim.x) sm[i] += sm[i + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

void dot(const double* a, const double* b, int64_t n, double* out, double* part, cudaStream_t s)
{
    k_dot_part<<<DOT_BLOCKS, NT, 0, s>>>(a, b, n, part); note_launch();
    k_dot_final<<<1, 256, 0, s>>>(part, out); note_launch();
    HM_LAUNCH("dot");
}

// r = b - q; p = r
__global__ void k_cg_init(const double* __restrict__ b, const double* __restrict__ q, int64_t n,
                          double* __restrict__ r, double* __restrict__ p)
{
    int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i < n) {
        double v = b[i] - q[i];
        r[i] = v;
        p[i] = v;
    }
}

// alpha = rr / pq; x += alpha p; r -= alpha q   (scalars on the device)
__global__ void k_cg_xr(const double* __restrict__ sc, const double* __restrict__ p,
                        const double* __restrict__ q, int64_t n, double* __restrict__ x,
                        double* __restrict__ r)
{
    int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i >= n) return;
    const double alpha = sc[0] / sc[1];
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
}

// beta = rr_new / rr; p = r + beta p
__global__ void k_cg_p(const double* __restrict__ sc, const double* __restrict__ r, int64_t n,
                       double* __restrict__ p)
{
    int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i >= n) return;
    const double beta = sc[2] / sc[0];
    p[i] = r[i] + beta * p[i];
}


__global__ void k_fill_i32(int32_t* __restrict__ p, int64_t n, int32_t v)
{
    int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

void fill_block_sets(hm_handle_s& h)
{
    h.adm_set.alloc(std::max<int64_t>(h.n_adm, 1), h.stream);
    h.dense_set.alloc(std::max<int64_t>(h.n_dense, 1), h.stream);
    int64_t a = 0, d = 0;
    for (size_t q = 0; q < h.sets.size(); ++q) {
        const SetStructure& S = h.sets[q];
        if (S.n_adm) k_fill_i32<<<grid_for(S.n_adm), NT, 0, h.stream>>>(h.adm_set.p + a, S.n_adm, (int)q); note_launch();
        if (S.n_dense)
            k_fill_i32<<<grid_for(S.n_dense), NT, 0, h.stream>>>(h.dense_set.p + d, S.n_dense, (int)q); note_launch();
        a += S.n_adm;
        d += S.n_dense;
    }
    HM_LAUNCH("block sets");
}

void add_perm_offsets(hm_handle_s& h)
{
    for (const SetStructure& S : h.sets)
        if (S.row0)
            k_add_offset<<<grid_for(S.N), NT, 0, h.stream>>>(h.perm.p + S.row0, S.N, S.row0); note_launch();
    HM_LAUNCH("perm offsets");
}

namespace {

// y (N1 entries per vector) = A_{phi, Y1 x Y2} x (N2 entries per vector):
// each x goes into set 1's part of a staging vector whose set 0 part stays
// zero, the square product runs on it (its blocks read columns of set 1 and
// its tiles are the rows of set 0 only), and set 0's part of the result is y.
void rect_matvec(hm_handle_s& h, const double* x, double* y, int nrhs, cudaStream_t s)
{
    const int64_t N = h.Ntot, N1 = h.n_rows, N2 = h.n_cols;
    if (!h.rxbuf.p) {
        h.rxbuf.alloc(N, h.stream);
        h.rybuf.alloc(N, h.stream);
        HM_CUDA(cudaMemsetAsync(h.rxbuf.p, 0, N * sizeof(double), h.stream));
        HM_CUDA(cudaMemsetAsync(h.rybuf.p, 0, N * sizeof(double), h.stream));
        HM_CUDA(cudaStreamSynchronize(h.stream));
    }
    for (int r = 0; r < nrhs; ++r) {
        copy_in(h.rxbuf.p + N1, x + (int64_t)r * N2, N2 * sizeof(double), s);
        if (h.opt.accumulate) copy_in(h.rybuf.p, y + (int64_t)r * N1, N1 * sizeof(double), s);
        if (h.opt.on_the_fly) np_matvec(h, h.rxbuf.p, h.rybuf.p, h.opt.accumulate, s);
        else mvp_run(h.plan, h.work, h.rxbuf.p, h.rybuf.p, h.opt.accumulate, s,
                     h.opt.profile ? &h.timer : nullptr);
        copy_out(y + (int64_t)r * N1, h.rybuf.p, N1 * sizeof(double), s);
    }
    if (!is_device_ptr(y)) HM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

// A product whose results go to host memory waits for them anyway; it then
// also reads the handle's status word (a bounded wait of the product that
// gave up) and reports it as HM_ETIMEOUT.
static void sync_and_check(hm_handle_s& h, cudaStream_t s)
{
    int st = 0;
    HM_CUDA(cudaMemcpyAsync(&st, h.status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    if (st) {
        HM_CUDA(cudaMemsetAsync(h.status.p, 0, sizeof(int), s));
        HM_CUDA(cudaStreamSynchronize(s));
        fail(HM_ETIMEOUT, "a bounded wait of the product gave up (status " + std::to_string(st) + ")");
    }
}

void matvec(hm_handle_s& h, const double* x, double* y, int nrhs, cudaStream_t s)
{
    if (h.opt.structure_only) fail(HM_EINVAL, "the handle was built with structure_only");
    if (h.rect) {
        rect_matvec(h, x, y, nrhs, s);
        return;
    }
    const int64_t N = h.Ntot;
    const bool xd = is_device_ptr(x), yd = is_device_ptr(y);
    if ((!xd || !yd) && !h.xbuf.p) {
        h.xbuf.alloc(N, h.stream);
        h.ybuf.alloc(N, h.stream);
        HM_CUDA(cudaStreamSynchronize(h.stream));
    }
    if (nrhs > 1 && !h.opt.on_the_fly && mvp_multi_fused(h.plan)) {
        // groups of up to MVP_NRC_MAX vectors share one pass over the stores
        constexpr int G = MVP_NRC_MAX;
        const bool grow_x = !xd && h.xbuf.n < (size_t)(N * G);
        const bool grow_y = !yd && h.ybuf.n < (size_t)(N * G);
        if (grow_x || grow_y) {
            HM_CUDA(cudaStreamSynchronize(s));   // earlier products may still read them
            if (grow_x) h.xbuf.alloc(N * G, h.stream);
            if (grow_y) h.ybuf.alloc(N * G, h.stream);
            HM_CUDA(cudaStreamSynchronize(h.stream));
        }
        for (int c = 0; c < nrhs; c += G) {
            const int nr = std::min(G, nrhs - c);
            const size_t bytes = (size_t)nr * N * sizeof(double);
            const double* xin = x + (int64_t)c * N;
            double* yout = y + (int64_t)c * N;
            if (!xd) {
                copy_in(h.xbuf.p, xin, bytes, s);
                xin = h.xbuf.p;
            }
            if (!yd) {
                if (h.opt.accumulate) copy_in(h.ybuf.p, yout, bytes, s);
                yout = h.ybuf.p;
            }
            mvp_run_multi(h.plan, h.work, xin, yout, nr, h.opt.accumulate, s);
            if (!yd) copy_out(y + (int64_t)c * N, h.ybuf.p, bytes, s);
        }
        if (!yd) sync_and_check(h, s);
        return;
    }
    for (int r = 0; r < nrhs; ++r) {
        const double* xr = x + (int64_t)r * N;
        double* yr = y + (int64_t)r * N;
        const double* xin = xr;
        double* yout = yr;
        if (!xd) {
            copy_in(h.xbuf.p, xr, N * sizeof(double), s);
            xin = h.xbuf.p;
        }
        if (!yd) {
            if (h.opt.accumulate) copy_in(h.ybuf.p, yr, N * sizeof(double), s);
            yout = h.ybuf.p;
        }
        if (h.opt.on_the_fly) np_matvec(h, xin, yout, h.opt.accumulate, s);
        else mvp_run(h.plan, h.work, xin, yout, h.opt.accumulate, s, h.opt.profile ? &h.timer : nullptr);
        if (!yd) copy_out(yr, h.ybuf.p, N * sizeof(double), s);
    }
    if (!yd) sync_and_check(h, s);
}

void export_structure(hm_handle_s& h, uint64_t* codes, int64_t* perm, int64_t* adm,
                      int64_t* dense, int32_t* ranks)
{
    cudaStream_t s = h.stream;
    const int64_t N = h.Ntot;
    if (codes) copy_out(codes, h.codes.p, N * sizeof(uint64_t), s);
    if (perm) {
        std::vector<int64_t> p(N);
        HM_CUDA(cudaMemcpyAsync(p.data(), h.perm.p, N * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        // set-local indices (the stored permutation is absolute)
        for (const SetStructure& S : h.sets)
            for (int64_t i = 0; i < S.N; ++i) p[S.row0 + i] -= S.row0;
        copy_out(perm, p.data(), N * sizeof(int64_t), s);
    }
    auto pairs = [&](const DevBuf<int2>& src, int64_t n, int64_t* dst) {
        std::vector<int2> v(std::max<int64_t>(n, 1));
        if (n) HM_CUDA(cudaMemcpyAsync(v.data(), src.p, n * sizeof(int2), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> o(2 * std::max<int64_t>(n, 1));
        for (int64_t b = 0; b < n; ++b) {
            o[2 * b] = v[b].x;
            o[2 * b + 1] = v[b].y;
        }
        copy_out(dst, o.data(), 2 * n * sizeof(int64_t), s);
    };
    if (adm) pairs(h.adm_pairs, h.n_adm, adm);
    if (dense) pairs(h.dense_pairs, h.n_dense, dense);
    if (ranks && h.n_adm) copy_out(ranks, h.rank.p, h.n_adm * sizeof(int32_t), s);
    HM_CUDA(cudaStreamSynchronize(s));
}

void export_tree(hm_handle_s& h, int64_t* lo, int64_t* hi, double* bbmin, double* bbmax)
{
    cudaStream_t s = h.stream;
    const int64_t nn = h.n_nodes_tot;
    std::vector<int32_t> l(nn), u(nn);
    std::vector<double> a(3 * nn), b(3 * nn);
    HM_CUDA(cudaMemcpyAsync(l.data(), h.node_lo.p, nn * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(u.data(), h.node_hi.p, nn * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(a.data(), h.bmin.p, 3 * nn * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(b.data(), h.bmax.p, 3 * nn * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    const int d = h.sets[0].d;
    std::vector<int64_t> L(nn), H(nn);
    std::vector<double> A(d * nn), B(d * nn);
    for (int64_t v = 0; v < nn; ++v) {
        L[v] = l[v];
        H[v] = u[v];
        for (int i = 0; i < d; ++i) {
            A[v * d + i] = l[v] >= 0 ? a[v * 3 + i] : 0.0;
            B[v * d + i] = l[v] >= 0 ? b[v * 3 + i] : 0.0;
        }
    }
    if (lo) copy_out(lo, L.data(), nn * sizeof(int64_t), s);
    if (hi) copy_out(hi, H.data(), nn * sizeof(int64_t), s);
    if (bbmin) copy_out(bbmin, A.data(), d * nn * sizeof(double), s);
    if (bbmax) copy_out(bbmax, B.data(), d * nn * sizeof(double), s);
    HM_CUDA(cudaStreamSynchronize(s));
}

void export_factors(hm_handle_s& h, int64_t b, double* U, double* V, int* rank)
{
    if (b < 0 || b >= h.n_adm) fail(HM_EINVAL, "block index out of range");
    if (h.opt.structure_only) fail(HM_EINVAL, "the handle was built with structure_only");
    if (h.opt.on_the_fly) fail(HM_ENOTSUP, "an on-the-fly handle stores no factors");
    cudaStream_t s = h.stream;
    Blk B;
    int r = 0;
    uint64_t vp = 0;
    HM_CUDA(cudaMemcpyAsync(&B, h.ablk.p + b, sizeof(Blk), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(&r, h.rank.p + b, sizeof(int), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(&vp, h.Vptr.p + b, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    if (rank) *rank = r;
    const bool f64 = h.precision == HM_PREC_FP64;
    const size_t esz = f64 ? 8 : 4;
    auto to_double = [&](const std::vector<char>& raw, size_t cnt, double* out) {
        for (size_t e = 0; e < cnt; ++e)
            out[e] = f64 ? reinterpret_cast<const double*>(raw.data())[e]
                         : (double)reinterpret_cast<const float*>(raw.data())[e];
    };
    const int64_t nv = (int64_t)r * B.n;
    if (V && nv) {
        std::vector<char> raw(nv * esz);
        HM_CUDA(cudaMemcpy(raw.data(), (const void*)vp, nv * esz, cudaMemcpyDeviceToHost));
        std::vector<double> tmp(nv);
        to_double(raw, nv, tmp.data());
        copy_out(V, tmp.data(), nv * sizeof(double), s);
    }
    if (U && r) {
        const MvpLists& L = h.lists;
        if (h.h_lr_ent.empty() && L.n_lr > 0) {
            h.h_lr_ent.resize(L.n_lr);
            h.h_lr_desc.resize(L.n_lr);
            h.h_lr_tile.resize(L.n_lr);
            h.h_tile_m.resize(h.n_tiles);
            HM_CUDA(cudaMemcpy(h.h_lr_ent.data(), L.lr_ent.p, L.n_lr * sizeof(int2), cudaMemcpyDeviceToHost));
            HM_CUDA(cudaMemcpy(h.h_lr_desc.data(), L.lr_desc.p, L.n_lr * sizeof(LrDesc), cudaMemcpyDeviceToHost));
            HM_CUDA(cudaMemcpy(h.h_lr_tile.data(), L.lr_tile.p, L.n_lr * sizeof(int32_t), cudaMemcpyDeviceToHost));
            HM_CUDA(cudaMemcpy(h.h_tile_m.data(), h.tile_m.p, h.n_tiles * sizeof(int32_t), cudaMemcpyDeviceToHost));
        }
        std::vector<double> tmp((size_t)r * B.m, 0.0);
        for (int64_t e = 0; e < L.n_lr; ++e) {
            if (h.h_lr_ent[e].x != b) continue;
            const int rows = h.h_tile_m[h.h_lr_tile[e]];
            const int ld = slice_ld(rows);
            const int rowoff = h.h_lr_ent[e].y;
            std::vector<char> raw((size_t)r * ld * esz);
            HM_CUDA(cudaMemcpy(raw.data(), h.ustore.p + h.h_lr_desc[e].uoff * esz, raw.size(),
                               cudaMemcpyDeviceToHost));
            std::vector<double> sl((size_t)r * rows);
            to_double(raw, sl.size(), sl.data());
            for (int l = 0; l < r; ++l)
                for (int i = 0; i < rows; ++i)
                    tmp[(size_t)l * B.m + rowoff + i] = sl[(size_t)l * ld + i];
        }
        copy_out(U, tmp.data(), tmp.size() * sizeof(double), s);
    }
    HM_CUDA(cudaStreamSynchronize(s));
}

// q = (H + sigma^2 I) p on device vectors, whatever the storage mode.
void apply_operator(hm_handle_s& h, const double* p, double* q, cudaStream_t s)
{
    if (h.opt.on_the_fly) np_matvec(h, p, q, 0, s);
    else mvp_run(h.plan, h.work, p, q, 0, s);
}

void cg_solve(hm_handle_s& h, const double* b, double* x, double rtol, int maxit, int* iters,
              double* relres)
{
    if (h.rect) fail(HM_EINVAL, "CG needs a square matrix (one set for rows and columns)");
    cudaStream_t s = h.stream;
    const int64_t n = h.Ntot;
    DevBuf<double> bd(n, s), xd(n, s), r(n, s), p(n, s), q(n, s), part(DOT_BLOCKS, s), sc(4, s);
    copy_in(bd.p, b, n * sizeof(double), s);
    copy_in(xd.p, x, n * sizeof(double), s);
    // sc[0] = rr, sc[1] = pq, sc[2] = rr_new, sc[3] = bb
    apply_operator(h, xd.p, q.p, s);
    k_cg_init<<<grid_for(n), NT, 0, s>>>(bd.p, q.p, n, r.p, p.p); note_launch();
    dot(bd.p, bd.p, n, sc.p + 3, part.p, s);
    dot(r.p, r.p, n, sc.p, part.p, s);
    double hs[4];
    HM_CUDA(cudaMemcpyAsync(hs, sc.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    double bn = std::sqrt(hs[3]);
    if (bn == 0.0) bn = 1.0;
    double rr = hs[0];
    int it = 0;
    while (it < maxit && std::sqrt(rr) / bn > rtol) {
        apply_operator(h, p.p, q.p, s);
        dot(p.p, q.p, n, sc.p + 1, part.p, s);
        k_cg_xr<<<grid_for(n), NT, 0, s>>>(sc.p, p.p, q.p, n, xd.p, r.p); note_launch();
        dot(r.p, r.p, n, sc.p + 2, part.p, s);
        k_cg_p<<<grid_for(n), NT, 0, s>>>(sc.p, r.p, n, p.p); note_launch();
        double got[3];
        HM_CUDA(cudaMemcpyAsync(sc.p, sc.p + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
        HM_CUDA(cudaMemcpyAsync(got, sc.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        rr = got[2];
        ++it;
        // p^T (H + sigma^2 I) p <= 0: the operator is not positive definite
        // along p (its approximation error exceeds the diagonal shift), and
        // the iteration has no meaning beyond this point
        if (!(got[1] > 0.0)) {
            if (iters) *iters = it;
            if (relres) *relres = std::sqrt(rr) / bn;
            fail(HM_EINVAL, "CG: p^T (H + sigma^2 I) p <= 0 at iteration " + std::to_string(it) +
                                ": the H-matrix plus sigma^2 I is not positive definite");
        }
    }
    copy_out(x, xd.p, n * sizeof(double), s);
    HM_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = std::sqrt(rr) / bn;
}

}  // namespace hm

using namespace hm;

extern "C" {

hm_batch hm_build_batch(int nsets, const double* points_all, const int64_t* N, const int* d,
                        int kernel, const double* params, int leaf_size, double eta,
                        double aca_eps, const hm_options* opt, int* status)
{
    set_error("");
    try {
        if (!N || !d) fail(HM_EINVAL, "null size arrays");
        hm_options o;
        hm_options_default(&o);
        if (opt) o = *opt;
        std::unique_ptr<hm_batch_s> b(new hm_batch_s());
        build_sets(b->h, nsets, points_all, N, d, kernel, params, leaf_size, eta, aca_eps, o);
        b->set_n.assign(N, N + nsets);
        b->set_d.assign(d, d + nsets);
        if (status) *status = HM_OK;
        return b.release();
    } catch (const std::exception& e) {
        int st = to_status(e);
        if (status) *status = st;
        return nullptr;
    }
}

int hm_matvec_batch(hm_batch b, const double* x_all, double* y_all)
{
    set_error("");
    try {
        if (!b || !x_all || !y_all) fail(HM_EINVAL, "null argument");
        matvec(b->h, x_all, y_all, 1, b->h.stream);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_batch_stats(hm_batch b, hm_stats* out)
{
    set_error("");
    if (!b || !out) {
        set_error("null argument");
        return HM_EINVAL;
    }
    return hm_get_stats(&b->h, out);
}

void hm_free_batch(hm_batch b)
{
    if (!b) return;
    try {
        cudaStream_t s = b->h.stream;
        delete b;
        cudaStreamSynchronize(s);
    } catch (...) {
    }
}

}  // extern "C"
