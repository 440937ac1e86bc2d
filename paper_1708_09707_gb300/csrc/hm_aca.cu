// hm_aca.cu -- batched adaptive cross approximation (Alg. 2, Sec. 5.4.1).
//
// Every admissible leaf is compressed independently; instead of the paper's
// batch-wide vote (all blocks iterate until the slowest one stops), each
// block stops on its own:
//  * blocks with m, n <= 32*MAXR are handled by one warp each: a lane owns
//    rows lane + 32t and columns lane + 32t, the residual column and row live
//    in registers, pivot searches and norms are warp-shuffle reductions;
//  * larger blocks get one CTA or one thread-block cluster each, with the
//    residual vectors in the output factor columns.
// Readings of Alg. 2 (the same as the CPU oracle): first column 0; row pivot
// argmax |u^| (lowest index on ties); a column whose largest residual entry
// is <= eps0 * max |A(:,j)| is rejected and the lowest unused column is tried;
// the next column is argmax over unused columns of |v_r|; ||S_r||_F^2 is
// updated by S2 += 2 sum_l (u.u_l)(v_l.v) + |u|^2 |v|^2; the rule
// |u||v| <= eps (1-aca_eta)/(1+eps) sqrt(S2) stops (eps <= 0: fixed rank).
// The norms, S2 and the stopping test are always accumulated in double.
#include <cooperative_groups.h>

#include "hm_kernel_fn.cuh"

namespace hm {

namespace {

constexpr int WARP_NT = 128;   // threads per CTA of the warp kernel
constexpr int CTA_NT = 256;
constexpr int CTA_WARPS = CTA_NT / 32;
constexpr int KBUF = 128;      // largest supported k_cap
constexpr int REJ_RUN = 4;     // rejected columns in a row that end a block

template <class R, int KERN, int MAXR>
__global__ void __launch_bounds__(WARP_NT)
k_aca_warp(KernelParams kp, DeviceCoords X, AcaArgs a, const uint32_t* __restrict__ order,
           int64_t nblocks, double thr)
{
    const int64_t wid = ((int64_t)blockIdx.x * WARP_NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= nblocks) return;
    const uint32_t b = order[wid];
    const Blk B = a.blk[b];
    const int m = B.m, n = B.n;
    const int kres = a.kres[b];
    int kmax = min(kres, min(m, n));
    R* __restrict__ U = reinterpret_cast<R*>(a.Uptr[b]);
    R* __restrict__ V = reinterpret_cast<R*>(a.Vptr[b]);
    const R c = kconst<R>(kp);
    const R eps0 = (R)a.eps0;

    R acc[MAXR];
    R vv[MAXR];
    unsigned used = 0;
    int r = 0, j = 0, rej = 0, run = 0;
    bool converged = false;
    double S2 = 0.0;
    const int limit = kmax + n + 1;

    for (int it = 0; r < kmax; ++it) {
        if (it > limit) {
            if (lane == 0) atomicOr(a.status, 1);
            break;
        }
        // residual column u^ = A(:, j) - sum_{l<r} u_l (v_l)_j
        if ((j & 31) == lane) used |= 1u << (j >> 5);
        const Pt<R> pj = load_pt<R>(X, B.col0 + j);
        R amax = 0;
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int i = lane + 32 * t;
            R v = 0;
            if (i < m) {
                v = phi<KERN>(dist2(load_pt<R>(X, B.row0 + i), pj), c);
                amax = max(amax, fabs(v));
            }
            acc[t] = v;
        }
        for (int l0 = 0; l0 < r; l0 += 32) {
            const R vjc = (l0 + lane < r) ? V[(int64_t)(l0 + lane) * n + j] : R(0);
            const int lend = min(r - l0, 32);
            for (int l = 0; l < lend; ++l) {
                const R vjl = __shfl_sync(0xffffffffu, vjc, l);
                const R* Ul = U + (int64_t)(l0 + l) * m;
#pragma unroll
                for (int t = 0; t < MAXR; ++t) {
                    const int i = lane + 32 * t;
                    if (i < m) acc[t] -= Ul[i] * vjl;
                }
            }
        }
        R best = -1;
        int bi = 0x7fffffff;
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int i = lane + 32 * t;
            if (i < m && fabs(acc[t]) > best) {
                best = fabs(acc[t]);
                bi = i;
            }
        }
        warp_argmax(best, bi);
        amax = warp_max(amax);
        if (!(best > eps0 * amax)) {
            // column already represented: take the lowest unused column,
            // or stop after REJ_RUN rejections in a row
            ++rej;
            if (++run >= REJ_RUN) {
                converged = true;
                break;
            }
            int cand = 0x7fffffff;
#pragma unroll
            for (int t = 0; t < MAXR; ++t) {
                const int jj = lane + 32 * t;
                if (jj < n && !((used >> t) & 1u)) {
                    cand = jj;
                    break;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
            if (cand == 0x7fffffff) {
                converged = true;
                break;
            }
            j = cand;
            continue;
        }
        run = 0;
        // u_r = u^ / u^_{i_r}
        R mine = 0;
#pragma unroll
        for (int t = 0; t < MAXR; ++t)
            if (t == (bi >> 5)) mine = acc[t];
        const R piv = __shfl_sync(0xffffffffu, mine, bi & 31);
        R* __restrict__ Ur = U + (int64_t)r * m;
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int i = lane + 32 * t;
            if (i < m) {
                acc[t] = acc[t] / piv;
                Ur[i] = acc[t];
            }
        }
        // residual row v = A(i_r, :)^T - sum_{l<r} (u_l)_{i_r} v_l
        const Pt<R> pi = load_pt<R>(X, B.row0 + bi);
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int jj = lane + 32 * t;
            vv[t] = (jj < n) ? phi<KERN>(dist2(pi, load_pt<R>(X, B.col0 + jj)), c) : R(0);
        }
        for (int l0 = 0; l0 < r; l0 += 32) {
            const R uic = (l0 + lane < r) ? U[(int64_t)(l0 + lane) * m + bi] : R(0);
            const int lend = min(r - l0, 32);
            for (int l = 0; l < lend; ++l) {
                const R uil = __shfl_sync(0xffffffffu, uic, l);
                const R* Vl = V + (int64_t)(l0 + l) * n;
#pragma unroll
                for (int t = 0; t < MAXR; ++t) {
                    const int jj = lane + 32 * t;
                    if (jj < n) vv[t] -= uil * Vl[jj];
                }
            }
        }
        R* __restrict__ Vr = V + (int64_t)r * n;
        double nu2 = 0.0, nv2 = 0.0;
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int i = lane + 32 * t;
            if (i < n) Vr[i] = vv[t];
            if (i < m) nu2 += (double)acc[t] * (double)acc[t];
            if (i < n) nv2 += (double)vv[t] * (double)vv[t];
        }
        nu2 = warp_sum(nu2);
        nv2 = warp_sum(nv2);
        // cross terms (u_r . u_l)(v_l . v_r)
        double cross = 0.0;
        for (int l = 0; l < r; ++l) {
            const R* Ul = U + (int64_t)l * m;
            const R* Vl = V + (int64_t)l * n;
            R du = 0, dv = 0;
#pragma unroll
            for (int t = 0; t < MAXR; ++t) {
                const int i = lane + 32 * t;
                if (i < m) du += acc[t] * Ul[i];
                if (i < n) dv += Vl[i] * vv[t];
            }
            double ddu = warp_sum((double)du);
            double ddv = warp_sum((double)dv);
            cross += ddu * ddv;
        }
        S2 += 2.0 * cross + nu2 * nv2;
        ++r;
        if (thr >= 0.0 && sqrt(nu2) * sqrt(nv2) <= thr * sqrt(fmax(S2, 0.0))) {
            converged = true;
            break;
        }
        if (r >= kmax) break;
        // next column: largest |v_r| over unused columns
        R bv = -1;
        int bj = 0x7fffffff;
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int jj = lane + 32 * t;
            if (jj < n && !((used >> t) & 1u) && fabs(vv[t]) > bv) {
                bv = fabs(vv[t]);
                bj = jj;
            }
        }
        warp_argmax(bv, bj);
        if (bj == 0x7fffffff) {
            converged = true;
            break;
        }
        j = bj;
    }
    if (lane == 0) {
        a.rank[b] = r;
        a.nrej[b] = rej;
        const int full = min(a.k_cap, min(m, n));
        int f = 0;
        if (!converged && r >= kmax) {
            if (kres < full) f |= 1;   // reservation too small: re-run
            else f |= 2;               // hit the rank cap
        }
        a.flags[b] = f;
    }
}

// --------------------------------------------------------------------------
// Large blocks: one CTA or one thread-block cluster of CS CTAs per block
// (CS = 1, 4 or 8). The rows and columns of the block are dealt round-robin
// to all CS * CTA_NT threads; every reduction (pivot search, norms, cross
// terms, next column) first reduces inside each CTA, then every CTA reads the
// partials of all CTAs of its cluster from distributed shared memory in rank
// order, so all CTAs reach identical decisions and follow the same control
// flow. Partials are double-buffered, so one cluster barrier per reduction
// suffices. The block's used-column bitmap lives in global memory.
// --------------------------------------------------------------------------
struct ClPart {
    double best, bval, amax;   // column pivot: |u^|, u^ at the pivot, max |A(:,j)|
    int bi, cand, vbj, pad;
    double nu2, nv2, vbest;
    double du[KBUF], dv[KBUF];
};

struct ClShared {
    ClPart part[2];
    double wl[CTA_WARPS][KBUF];   // per-warp partial dots
    double wm[CTA_WARPS][KBUF];
    double ws[CTA_WARPS][4];
    int wi[CTA_WARPS][2];
    double bc[4];                 // broadcast: reduced values
    int bci[2];
};

template <class R, int KERN>
__global__ void __launch_bounds__(CTA_NT)
k_aca_cluster(KernelParams kp, DeviceCoords X, AcaArgs a, const uint32_t* __restrict__ order,
              int64_t nblocks, double thr, uint32_t* __restrict__ usedpool, int64_t used_words)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks();
    const int crank = (int)cl.block_rank();
    __shared__ R sg[KBUF];
    __shared__ ClShared sh;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int gt = crank * CTA_NT + tid, GT = CS * CTA_NT;
    const int64_t cid = blockIdx.x / CS, ncl = gridDim.x / CS;
    uint32_t* used = usedpool + cid * used_words;
    const R c = kconst<R>(kp);
    const R eps0 = (R)a.eps0;
    int ph = 0;

    for (int64_t q = cid; q < nblocks; q += ncl) {
        const uint32_t b = order[q];
        const Blk B = a.blk[b];
        const int m = B.m, n = B.n;
        const int kres = a.kres[b];
        const int kmax = min(kres, min(m, n));
        R* __restrict__ U = reinterpret_cast<R*>(a.Uptr[b]);
        R* __restrict__ V = reinterpret_cast<R*>(a.Vptr[b]);
        const int words = (n + 31) / 32;
        for (int k = gt; k < words; k += GT) used[k] = 0u;
        cl.sync();

        int r = 0, j = 0, rej = 0, run = 0;
        bool converged = false;
        double S2 = 0.0;
        const int limit = kmax + n + 1;
        for (int it = 0; r < kmax; ++it) {
            if (it > limit) {
                if (gt == 0) atomicOr(a.status, 1);
                break;
            }
            if (gt == 0) used[j >> 5] |= 1u << (j & 31);
            if (tid < r) sg[tid] = V[(int64_t)tid * n + j];
            __syncthreads();
            // residual column and its pivot
            const Pt<R> pj = load_pt<R>(X, B.col0 + j);
            R* __restrict__ Ur = U + (int64_t)r * m;
            R best = -1, amax = 0, bval = 0;
            int bi = 0x7fffffff;
            for (int i = gt; i < m; i += GT) {
                R v = phi<KERN>(dist2(load_pt<R>(X, B.row0 + i), pj), c);
                amax = max(amax, fabs(v));
                for (int l = 0; l < r; ++l) v -= U[(int64_t)l * m + i] * sg[l];
                Ur[i] = v;
                if (fabs(v) > best) {
                    best = fabs(v);
                    bi = i;
                    bval = v;
                }
            }
            {
                // warp then CTA argmax carrying the signed value
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    R ob = __shfl_xor_sync(0xffffffffu, best, o);
                    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    R ov = __shfl_xor_sync(0xffffffffu, bval, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                        bval = ov;
                    }
                }
                amax = warp_max(amax);
                if (lane == 0) {
                    sh.ws[w][0] = (double)best;
                    sh.ws[w][1] = (double)bval;
                    sh.ws[w][2] = (double)amax;
                    sh.wi[w][0] = bi;
                }
                __syncthreads();
                if (tid == 0) {
                    double B0 = sh.ws[0][0], V0 = sh.ws[0][1], A0 = sh.ws[0][2];
                    int I0 = sh.wi[0][0];
                    for (int k = 1; k < CTA_WARPS; ++k) {
                        if (sh.ws[k][0] > B0 || (sh.ws[k][0] == B0 && sh.wi[k][0] < I0)) {
                            B0 = sh.ws[k][0];
                            V0 = sh.ws[k][1];
                            I0 = sh.wi[k][0];
                        }
                        A0 = fmax(A0, sh.ws[k][2]);
                    }
                    sh.part[ph].best = B0;
                    sh.part[ph].bval = V0;
                    sh.part[ph].amax = A0;
                    sh.part[ph].bi = I0;
                }
                cl.sync();
                if (tid == 0) {
                    double B0 = -1, V0 = 0, A0 = 0;
                    int I0 = 0x7fffffff;
                    for (int k = 0; k < CS; ++k) {
                        const ClPart* P = cl.map_shared_rank(&sh.part[ph], k);
                        if (P->best > B0 || (P->best == B0 && P->bi < I0)) {
                            B0 = P->best;
                            V0 = P->bval;
                            I0 = P->bi;
                        }
                        A0 = fmax(A0, P->amax);
                    }
                    sh.bc[0] = B0;
                    sh.bc[1] = V0;
                    sh.bc[2] = A0;
                    sh.bci[0] = I0;
                }
                ph ^= 1;
                __syncthreads();
                best = (R)sh.bc[0];
                bval = (R)sh.bc[1];
                amax = (R)sh.bc[2];
                bi = sh.bci[0];
                __syncthreads();
            }
            if (!(best > eps0 * amax)) {
                ++rej;
                if (++run >= REJ_RUN) {
                    converged = true;
                    break;
                }
                // lowest unused column over the whole cluster
                int cand = 0x7fffffff;
                for (int k = gt; k < words; k += GT) {
                    uint32_t free_bits = ~used[k];
                    if (k == words - 1 && (n & 31)) free_bits &= (1u << (n & 31)) - 1u;
                    if (free_bits) {
                        cand = k * 32 + __ffs(free_bits) - 1;
                        break;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
                if (lane == 0) sh.wi[w][1] = cand;
                __syncthreads();
                if (tid == 0) {
                    int cm = 0x7fffffff;
                    for (int k = 0; k < CTA_WARPS; ++k) cm = min(cm, sh.wi[k][1]);
                    sh.part[ph].cand = cm;
                }
                cl.sync();
                if (tid == 0) {
                    int cm = 0x7fffffff;
                    for (int k = 0; k < CS; ++k) cm = min(cm, cl.map_shared_rank(&sh.part[ph], k)->cand);
                    sh.bci[1] = cm;
                }
                ph ^= 1;
                __syncthreads();
                cand = sh.bci[1];
                __syncthreads();
                if (cand == 0x7fffffff || cand >= n) {
                    converged = true;
                    break;
                }
                j = cand;
                continue;
            }
            run = 0;
            const R piv = bval;
            if (tid < r) sg[tid] = U[(int64_t)tid * m + bi];
            __syncthreads();
            // residual row, scaled column, norms and next-column candidates
            const Pt<R> pi = load_pt<R>(X, B.row0 + bi);
            R* __restrict__ Vr = V + (int64_t)r * n;
            double nv2 = 0.0, nu2 = 0.0;
            R vb = -1;
            int vbj = 0x7fffffff;
            for (int jj = gt; jj < n; jj += GT) {
                R v = phi<KERN>(dist2(pi, load_pt<R>(X, B.col0 + jj)), c);
                for (int l = 0; l < r; ++l) v -= sg[l] * V[(int64_t)l * n + jj];
                Vr[jj] = v;
                nv2 += (double)v * (double)v;
                if (!((used[jj >> 5] >> (jj & 31)) & 1u) && fabs(v) > vb) {
                    vb = fabs(v);
                    vbj = jj;
                }
            }
            for (int i = gt; i < m; i += GT) {
                const R u = Ur[i] / piv;
                Ur[i] = u;
                nu2 += (double)u * (double)u;
            }
            for (int l = 0; l < r; ++l) {
                const R* Ul = U + (int64_t)l * m;
                const R* Vl = V + (int64_t)l * n;
                R du = 0, dv = 0;
                for (int i = gt; i < m; i += GT) du += Ur[i] * Ul[i];
                for (int jj = gt; jj < n; jj += GT) dv += Vl[jj] * Vr[jj];
                const double ddu = warp_sum((double)du), ddv = warp_sum((double)dv);
                if (lane == 0) {
                    sh.wl[w][l] = ddu;
                    sh.wm[w][l] = ddv;
                }
            }
            nu2 = warp_sum(nu2);
            nv2 = warp_sum(nv2);
            warp_argmax(vb, vbj);
            if (lane == 0) {
                sh.ws[w][0] = nu2;
                sh.ws[w][1] = nv2;
                sh.ws[w][2] = (double)vb;
                sh.wi[w][0] = vbj;
            }
            __syncthreads();
            {
                ClPart& P = sh.part[ph];
                if (tid < r) {
                    double su = 0.0, sv = 0.0;
                    for (int k = 0; k < CTA_WARPS; ++k) {
                        su += sh.wl[k][tid];
                        sv += sh.wm[k][tid];
                    }
                    P.du[tid] = su;
                    P.dv[tid] = sv;
                }
                if (tid == 0) {
                    double a0 = 0.0, a1 = 0.0, B0 = -1.0;
                    int I0 = 0x7fffffff;
                    for (int k = 0; k < CTA_WARPS; ++k) {
                        a0 += sh.ws[k][0];
                        a1 += sh.ws[k][1];
                        if (sh.ws[k][2] > B0 || (sh.ws[k][2] == B0 && sh.wi[k][0] < I0)) {
                            B0 = sh.ws[k][2];
                            I0 = sh.wi[k][0];
                        }
                    }
                    P.nu2 = a0;
                    P.nv2 = a1;
                    P.vbest = B0;
                    P.vbj = I0;
                }
            }
            cl.sync();
            if (w == 0) {
                // cross term sum_l (sum_ranks du_l)(sum_ranks dv_l), in rank order
                double cr = 0.0;
                for (int l0 = 0; l0 < r; l0 += 32) {
                    const int l = l0 + lane;
                    double su = 0.0, sv = 0.0;
                    if (l < r)
                        for (int k = 0; k < CS; ++k) {
                            const ClPart* P = cl.map_shared_rank(&sh.part[ph], k);
                            su += P->du[l];
                            sv += P->dv[l];
                        }
                    cr += warp_sum(su * sv);
                }
                if (lane == 0) {
                    double a0 = 0.0, a1 = 0.0, B0 = -1.0;
                    int I0 = 0x7fffffff;
                    for (int k = 0; k < CS; ++k) {
                        const ClPart* P = cl.map_shared_rank(&sh.part[ph], k);
                        a0 += P->nu2;
                        a1 += P->nv2;
                        if (P->vbest > B0 || (P->vbest == B0 && P->vbj < I0)) {
                            B0 = P->vbest;
                            I0 = P->vbj;
                        }
                    }
                    sh.bc[0] = a0;
                    sh.bc[1] = a1;
                    sh.bc[2] = cr;
                    sh.bci[0] = I0;
                }
            }
            ph ^= 1;
            __syncthreads();
            const double NU2 = sh.bc[0], NV2 = sh.bc[1], cross = sh.bc[2];
            const int nj = sh.bci[0];
            __syncthreads();
            S2 += 2.0 * cross + NU2 * NV2;
            ++r;
            if (thr >= 0.0 && sqrt(NU2) * sqrt(NV2) <= thr * sqrt(fmax(S2, 0.0))) {
                converged = true;
                break;
            }
            if (r >= kmax) break;
            if (nj == 0x7fffffff) {
                converged = true;
                break;
            }
            j = nj;
        }
        if (gt == 0) {
            a.rank[b] = r;
            a.nrej[b] = rej;
            const int full = min(a.k_cap, min(m, n));
            int f = 0;
            if (!converged && r >= kmax) f |= (kres < full) ? 1 : 2;
            a.flags[b] = f;
        }
        cl.sync();
    }
}

template <class R, int KERN>
void launch_all(const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                const uint32_t* order, int64_t n, int cls, int64_t max_n, cudaStream_t s)
{
    const double thr = (a.eps > 0.0) ? a.eps * (1.0 - a.aca_eta) / (1.0 + a.eps) : -1.0;
    const unsigned wgrid = (unsigned)ceil_div(n * 32, WARP_NT);
    switch (cls) {
    case 0: k_aca_warp<R, KERN, 2><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr); note_launch(); break;
    case 1: k_aca_warp<R, KERN, 4><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr); note_launch(); break;
    case 2: k_aca_warp<R, KERN, 8><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr); note_launch(); break;
    case 3: k_aca_warp<R, KERN, 16><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr); note_launch(); break;
    default: {
        const int cs = cls == 4 ? 1 : (cls == 5 ? 4 : 8);
        int occ = 0;
        HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_aca_cluster<R, KERN>,
                                                              CTA_NT, 0));
        int64_t nclusters = std::min<int64_t>(n, std::max<int64_t>(1, (int64_t)std::max(occ, 1) *
                                                                         num_sms() / cs));
        const int64_t words = ceil_div(max_n, 32);
        DevBuf<uint32_t> usedpool((size_t)(nclusters * words), s);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nclusters * cs));
        cfg.blockDim = dim3(CTA_NT);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        HM_CUDA(cudaLaunchKernelEx(&cfg, k_aca_cluster<R, KERN>, kp, X, a, order, n, thr,
                                   usedpool.p, words));
        note_launch();
        break;
    }
    }
    HM_LAUNCH("aca");
}


}  // namespace

void aca_run(int precision, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
             const uint32_t* order, int64_t n, int cls, int64_t max_n, cudaStream_t s)
{
    if (n <= 0) return;
    if (a.k_cap > KBUF) fail(HM_ENOTSUP, "k_cap above 128 is not supported");
    const bool f64 = precision == HM_PREC_FP64;
    if (kp.kernel == HM_GAUSSIAN) {
        if (f64) launch_all<double, HM_GAUSSIAN>(kp, X, a, order, n, cls, max_n, s);
        else launch_all<float, HM_GAUSSIAN>(kp, X, a, order, n, cls, max_n, s);
    } else {
        if (f64) launch_all<double, HM_MATERN32>(kp, X, a, order, n, cls, max_n, s);
        else launch_all<float, HM_MATERN32>(kp, X, a, order, n, cls, max_n, s);
    }
}

int aca_class_of(int m, int n)
{
    const int d = m > n ? m : n;
    for (int c = 0; c < ACA_NCLASS - 1; ++c)
        if (d <= kAcaClassDim[c]) return c;
    return ACA_NCLASS - 1;
}

}  // namespace hm
