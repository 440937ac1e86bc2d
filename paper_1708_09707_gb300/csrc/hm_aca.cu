// hm_aca.cu -- batched adaptive cross approximation (Alg. 2, Sec. 5.4.1).
//
// Every admissible leaf is compressed independently; instead of the paper's
// batch-wide vote (all blocks iterate until the slowest one stops), each
// block stops on its own:
//  * blocks with m, n <= 32*MAXR are handled by one warp each: a lane owns
//    rows lane + 32t and columns lane + 32t, the residual column and row live
//    in registers, pivot searches and norms are warp-shuffle reductions;
//  * larger blocks get one CTA each (persistent CTAs pull blocks from a
//    counter), with the residual vectors in the output factor columns.
// Readings of Alg. 2 (the same as the CPU oracle): first column 0; row pivot
// argmax |u^| (lowest index on ties); a column whose largest residual entry
// is <= eps0 * max |A(:,j)| is rejected and the lowest unused column is tried;
// the next column is argmax over unused columns of |v_r|; ||S_r||_F^2 is
// updated by S2 += 2 sum_l (u.u_l)(v_l.v) + |u|^2 |v|^2; the rule
// |u||v| <= eps (1-aca_eta)/(1+eps) sqrt(S2) stops (eps <= 0: fixed rank).
// The norms, S2 and the stopping test are always accumulated in double.
#include "hm_kernel_fn.cuh"

namespace hm {

namespace {

constexpr int WARP_NT = 128;   // threads per CTA of the warp kernel
constexpr int CTA_NT = 512;
constexpr int CTA_WARPS = CTA_NT / 32;
constexpr int KBUF = 128;      // largest supported k_cap

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
    int r = 0, j = 0, rej = 0;
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
            // column already represented: take the lowest unused column
            ++rej;
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
// One CTA per large block; persistent CTAs take blocks from a counter.
// --------------------------------------------------------------------------
struct CtaRed {
    double dsum[CTA_WARPS][2];
    double dl[CTA_WARPS][KBUF];
    double dm[CTA_WARPS][KBUF];
    float fbest[CTA_WARPS];
    double dbest[CTA_WARPS];
    int ibest[CTA_WARPS];
    double damax[CTA_WARPS];
};

template <class R>
__device__ __forceinline__ void cta_argmax(R val, int idx, R amax, CtaRed& red, R& out_val,
                                           int& out_idx, R& out_amax)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    warp_argmax(val, idx);
    amax = warp_max(amax);
    if (lane == 0) {
        red.dbest[w] = (double)val;
        red.ibest[w] = idx;
        red.damax[w] = (double)amax;
    }
    __syncthreads();
    double bv = red.dbest[0];
    int bi = red.ibest[0];
    double am = red.damax[0];
    for (int k = 1; k < CTA_WARPS; ++k) {
        double v = red.dbest[k];
        int i = red.ibest[k];
        if (v > bv || (v == bv && i < bi)) {
            bv = v;
            bi = i;
        }
        am = fmax(am, red.damax[k]);
    }
    __syncthreads();
    out_val = (R)bv;
    out_idx = bi;
    out_amax = (R)am;
}

template <class R, int KERN>
__global__ void __launch_bounds__(CTA_NT, 1)
k_aca_cta(KernelParams kp, DeviceCoords X, AcaArgs a, const uint32_t* __restrict__ order,
          int64_t nblocks, double thr, int* __restrict__ counter,
          uint32_t* __restrict__ usedpool, int64_t used_words)
{
    __shared__ R sg[KBUF];
    __shared__ CtaRed red;
    __shared__ int s_next;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    uint32_t* used = usedpool + (int64_t)blockIdx.x * used_words;
    const R c = kconst<R>(kp);
    const R eps0 = (R)a.eps0;

    for (;;) {
        if (tid == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int64_t q = s_next;
        __syncthreads();
        if (q >= nblocks) break;
        const uint32_t b = order[q];
        const Blk B = a.blk[b];
        const int m = B.m, n = B.n;
        const int kres = a.kres[b];
        const int kmax = min(kres, min(m, n));
        R* __restrict__ U = reinterpret_cast<R*>(a.Uptr[b]);
        R* __restrict__ V = reinterpret_cast<R*>(a.Vptr[b]);
        for (int k = tid; k < (n + 31) / 32; k += CTA_NT) used[k] = 0u;
        __syncthreads();

        int r = 0, j = 0, rej = 0;
        bool converged = false;
        double S2 = 0.0;
        const int limit = kmax + n + 1;
        for (int it = 0; r < kmax; ++it) {
            if (it > limit) {
                if (tid == 0) atomicOr(a.status, 1);
                break;
            }
            if (tid == 0) used[j >> 5] |= 1u << (j & 31);
            if (tid < r) sg[tid] = V[(int64_t)tid * n + j];
            __syncthreads();
            const Pt<R> pj = load_pt<R>(X, B.col0 + j);
            R* __restrict__ Ur = U + (int64_t)r * m;
            R best = -1, amax = 0;
            int bi = 0x7fffffff;
            for (int i = tid; i < m; i += CTA_NT) {
                R v = phi<KERN>(dist2(load_pt<R>(X, B.row0 + i), pj), c);
                amax = max(amax, fabs(v));
                for (int l = 0; l < r; ++l) v -= U[(int64_t)l * m + i] * sg[l];
                Ur[i] = v;
                if (fabs(v) > best) {
                    best = fabs(v);
                    bi = i;
                }
            }
            cta_argmax<R>(best, bi, amax, red, best, bi, amax);
            if (!(best > eps0 * amax)) {
                ++rej;
                // lowest unused column
                int cand = 0x7fffffff;
                for (int k = tid; k < (n + 31) / 32; k += CTA_NT) {
                    uint32_t free_bits = ~used[k];
                    if (k == (n - 1) / 32 && (n & 31)) free_bits &= (1u << (n & 31)) - 1u;
                    if (free_bits) {
                        cand = k * 32 + __ffs(free_bits) - 1;
                        break;
                    }
                }
                // all values equal: the argmax tie rule returns the lowest index
                R dummy = 0;
                R dv0 = 0;
                cta_argmax<R>(dv0, cand, dummy, red, dv0, cand, dummy);
                if (cand == 0x7fffffff || cand < 0 || cand >= n) {
                    converged = true;
                    break;
                }
                j = cand;
                continue;
            }
            // scale, gather U(i_r, l)
            const R piv = Ur[bi];
            __syncthreads();
            for (int i = tid; i < m; i += CTA_NT) Ur[i] = Ur[i] / piv;
            if (tid < r) sg[tid] = U[(int64_t)tid * m + bi];
            __syncthreads();
            const Pt<R> pi = load_pt<R>(X, B.row0 + bi);
            R* __restrict__ Vr = V + (int64_t)r * n;
            double nv2 = 0.0;
            for (int jj = tid; jj < n; jj += CTA_NT) {
                R v = phi<KERN>(dist2(pi, load_pt<R>(X, B.col0 + jj)), c);
                for (int l = 0; l < r; ++l) v -= sg[l] * V[(int64_t)l * n + jj];
                Vr[jj] = v;
                nv2 += (double)v * (double)v;
            }
            double nu2 = 0.0;
            for (int i = tid; i < m; i += CTA_NT) nu2 += (double)Ur[i] * (double)Ur[i];
            // per-warp partial dots for all l, one reduction across warps
            for (int l = 0; l < r; ++l) {
                const R* Ul = U + (int64_t)l * m;
                const R* Vl = V + (int64_t)l * n;
                R du = 0, dv = 0;
                for (int i = tid; i < m; i += CTA_NT) du += Ur[i] * Ul[i];
                for (int jj = tid; jj < n; jj += CTA_NT) dv += Vl[jj] * Vr[jj];
                double ddu = warp_sum((double)du), ddv = warp_sum((double)dv);
                if (lane == 0) {
                    red.dl[w][l] = ddu;
                    red.dm[w][l] = ddv;
                }
            }
            nu2 = warp_sum(nu2);
            nv2 = warp_sum(nv2);
            if (lane == 0) {
                red.dsum[w][0] = nu2;
                red.dsum[w][1] = nv2;
            }
            __syncthreads();
            double NU2 = 0.0, NV2 = 0.0, cross = 0.0;
            for (int k = 0; k < CTA_WARPS; ++k) {
                NU2 += red.dsum[k][0];
                NV2 += red.dsum[k][1];
            }
            for (int l = 0; l < r; ++l) {
                double du = 0.0, dv = 0.0;
                for (int k = 0; k < CTA_WARPS; ++k) {
                    du += red.dl[k][l];
                    dv += red.dm[k][l];
                }
                cross += du * dv;
            }
            __syncthreads();
            S2 += 2.0 * cross + NU2 * NV2;
            ++r;
            if (thr >= 0.0 && sqrt(NU2) * sqrt(NV2) <= thr * sqrt(fmax(S2, 0.0))) {
                converged = true;
                break;
            }
            if (r >= kmax) break;
            // next column: largest |v_r| over unused columns
            R bv = -1, dummy = 0;
            int bj = 0x7fffffff;
            for (int jj = tid; jj < n; jj += CTA_NT) {
                if ((used[jj >> 5] >> (jj & 31)) & 1u) continue;
                R v = fabs(Vr[jj]);
                if (v > bv) {
                    bv = v;
                    bj = jj;
                }
            }
            cta_argmax<R>(bv, bj, dummy, red, bv, bj, dummy);
            if (bj == 0x7fffffff) {
                converged = true;
                break;
            }
            j = bj;
        }
        if (tid == 0) {
            a.rank[b] = r;
            a.nrej[b] = rej;
            const int full = min(a.k_cap, min(m, n));
            int f = 0;
            if (!converged && r >= kmax) f |= (kres < full) ? 1 : 2;
            a.flags[b] = f;
        }
        __syncthreads();
    }
}

template <class R, int KERN>
void launch_all(const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                const uint32_t* order, int64_t n, int64_t max_dim, cudaStream_t s)
{
    // blocks are given grouped by size class: the caller passes the size
    // classes one at a time (max_dim is the class bound)
    const double thr = (a.eps > 0.0) ? a.eps * (1.0 - a.aca_eta) / (1.0 + a.eps) : -1.0;
    const unsigned wgrid = (unsigned)ceil_div(n * 32, WARP_NT);
    if (max_dim <= 64) {
        k_aca_warp<R, KERN, 2><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr);
    } else if (max_dim <= 128) {
        k_aca_warp<R, KERN, 4><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr);
    } else if (max_dim <= 256) {
        k_aca_warp<R, KERN, 8><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr);
    } else if (max_dim <= 512) {
        k_aca_warp<R, KERN, 16><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr);
    } else {
        int occ = 0;
        HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_aca_cta<R, KERN>, CTA_NT, 0));
        int64_t grid = std::min<int64_t>(n, (int64_t)std::max(occ, 1) * num_sms());
        int64_t words = ceil_div(max_dim, 32);
        DevBuf<uint32_t> usedpool((size_t)(grid * words), s);
        DevBuf<int> counter(1, s);
        HM_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(int), s));
        k_aca_cta<R, KERN><<<(unsigned)grid, CTA_NT, 0, s>>>(kp, X, a, order, n, thr, counter.p,
                                                            usedpool.p, words);
    }
    HM_LAUNCH("aca");
}

}  // namespace

void aca_run(int precision, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
             const uint32_t* order, int64_t n, int64_t max_dim, cudaStream_t s)
{
    if (n <= 0) return;
    if (a.k_cap > KBUF) fail(HM_ENOTSUP, "k_cap above 128 is not supported");
    const bool f64 = precision == HM_PREC_FP64;
    if (kp.kernel == HM_GAUSSIAN) {
        if (f64) launch_all<double, HM_GAUSSIAN>(kp, X, a, order, n, max_dim, s);
        else launch_all<float, HM_GAUSSIAN>(kp, X, a, order, n, max_dim, s);
    } else {
        if (f64) launch_all<double, HM_MATERN32>(kp, X, a, order, n, max_dim, s);
        else launch_all<float, HM_MATERN32>(kp, X, a, order, n, max_dim, s);
    }
}

}  // namespace hm
