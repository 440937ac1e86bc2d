// hm_aca_impl.cuh -- batched adaptive cross approximation (Alg. 2, Sec. 5.4.1):
// the kernel templates and their launchers. hm_aca.cu instantiates them for
// the Gaussian and Matern-3/2 kernels, hm_aca_k1.cu for the Matern kernel of
// order 1 (two translation units, compiled in parallel).
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
// is <= eps0 * max |A(:,j)| is rejected and the lowest unused column is tried
// (four rejections in a row end the block); the next column is the argmax
// over unused columns of the residual of a reference row (row 0, moved to the
// lowest row not yet used as pivot or reference once its residual is below
// tol sqrt(S2 / m), tol = eps, or eps0 in fixed-rank mode);
// ||S_r||_F^2 is updated by S2 += 2 sum_l (u.u_l)(v_l.v) + |u|^2 |v|^2; the
// rule |u||v| <= eps (1-aca_eta)/(1+eps) sqrt(S2) with the reference row
// resolved stops (eps <= 0: fixed rank).
//
// Mixed precision adds a global floor to both tests: S2 is replaced by
// max(S2, m n / N). Since ||A||_F >= sqrt(N) phi(0) with phi(0) = 1, blocks
// that meet the floored tests keep ||A - H||_F <= eps ||A||_F overall, while
// far blocks whose entries are far below float resolution (exp(-x) with
// x ~ 100 is subnormal in float) stop at rank 1 instead of fitting rounding
// noise up to the rank cap.
// The norms, S2 and the stopping test are accumulated in double across
// threads; inside a thread the float kernels keep their partials in float
// (compensated sums, exact maxima), since this GPU's double pipe runs at a
// small fraction of its float rate.
#pragma once

#include <cooperative_groups.h>

#include "hm_kernel_fn.cuh"

namespace hm {

namespace {

constexpr int WARP_NT = 128;   // threads per CTA of the warp kernel
constexpr int CTA_NT = 256;
constexpr int CTA_WARPS = CTA_NT / 32;
constexpr int KBUF = 128;      // largest supported k_cap
// Rejected columns in a row that end a block: four in double precision (the
// oracle's rule); two in float, where a rejected column's residual is
// already at float resolution relative to the column.
template <class T>
__host__ __device__ constexpr int rej_run()
{
    return sizeof(T) == 4 ? 2 : 4;
}
constexpr int UNR = 4;         // rows (columns) per thread whose loads are issued together
constexpr int LC = 4;          // ranks per batch of loads and dot products

// Warp sums of LC per-lane values (a reduce-scatter butterfly): afterwards
// the lanes L with scatter_elem(L) == e hold the total of value e, and lane
// scatter_writer(e) is the first of them.
template <class T>
__device__ __forceinline__ T warp_scatter(const T (&p)[LC])
{
    static_assert(LC == 4, "reduce-scatter of four values");
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8;
    T a2[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const T send = h16 ? p[e] : p[e + 2];
        const T keep = h16 ? p[e + 2] : p[e];
        a2[e] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    T a1 = (h8 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h8 ? a2[0] : a2[1], 8);
    a1 += __shfl_xor_sync(0xffffffffu, a1, 4);
    a1 += __shfl_xor_sync(0xffffffffu, a1, 2);
    a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
    return a1;
}
__device__ __forceinline__ int scatter_elem(int lane) { return (lane >> 3) & 3; }
__device__ __forceinline__ bool scatter_writer(int lane) { return (lane & 7) == 0; }

// The stopping rule of one ACA step, kept in double: ||S_r||_F^2 += 2 cross +
// |u_r|^2 |v_r|^2, then the rule |u_r|^2 |v_r|^2 <= thr^2 S2 and the
// reference-row limit rmax^2 <= tol^2 S2 / m, with S2 floored at floor2. In
// the float kernels the step's terms are formed in float and widened once, so
// a step costs nine double-pipe instructions, which matters on this GPU
// where the double pipe runs at a small fraction of the float rate.
struct StopState {
    double S2 = 0.0, floor2 = 0.0, rtol2_m = 0.0, thr2 = 0.0, rlim2 = 0.0;
    bool fixed_rank = false;
};

__device__ __forceinline__ void stop_step(StopState& st, const TSum<double>& nu2,
                                          const TSum<double>& nv2, double cross, double rmax,
                                          bool& resolved, bool& stop_ok)
{
    const double p = nu2.value() * nv2.value();
    st.S2 += 2.0 * cross + p;
    const double S2f = fmax(st.S2, st.floor2);
    st.rlim2 = st.rtol2_m * S2f;
    resolved = !(rmax * rmax > st.rlim2);
    stop_ok = !st.fixed_rank && p <= st.thr2 * S2f;
}

__device__ __forceinline__ void stop_step(StopState& st, const TSum<float>& nu2,
                                          const TSum<float>& nv2, float cross, float rmax,
                                          bool& resolved, bool& stop_ok)
{
    const float p = nu2.rvalue() * nv2.rvalue();
    st.S2 += (double)fmaf(2.f, cross, p);
    const double S2f = fmax(st.S2, st.floor2);
    st.rlim2 = st.rtol2_m * S2f;
    resolved = !((double)(rmax * rmax) > st.rlim2);
    stop_ok = !st.fixed_rank && (double)p <= st.thr2 * S2f;
}

// The reference-row limit alone (after the reference row moved).
__device__ __forceinline__ bool ref_resolved(const StopState& st, double rmax)
{
    return !(rmax * rmax > st.rlim2);
}
__device__ __forceinline__ bool ref_resolved(const StopState& st, float rmax)
{
    return !((double)(rmax * rmax) > st.rlim2);
}

// --------------------------------------------------------------------------
// One warp per block (m, n <= 32 MAXR). Lane l owns rows and columns
// l + 32 t, t < MAXR: the residual column, the residual row and the
// reference-row residual live in registers; used columns and seen rows are
// bit masks per lane.
// --------------------------------------------------------------------------
template <class R, int KERN, int MAXR>
__global__ void __launch_bounds__(WARP_NT, MAXR <= 2 ? 8 : (MAXR <= 4 ? 6 : 4))
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
    const int kmax = min(kres, min(m, n));
    R* __restrict__ U = reinterpret_cast<R*>(a.Uptr[b]);
    R* __restrict__ V = reinterpret_cast<R*>(a.Vptr[b]);
    const R c = kconst<R>(kp);
    const R eps0 = (R)a.eps0;
    const double rtol = a.eps > 0.0 ? a.eps : a.eps0;
    const double floor2 = a.bset ? (double)m * (double)n / (double)a.set_n[a.bset[b]] : 0.0;

    // ranks whose loads are issued together
    constexpr int WB = MAXR <= 4 ? 4 : (MAXR <= 8 ? 2 : 1);
    R acc[MAXR], vv[MAXR];
    Resid<R> res[MAXR], rr[MAXR];   // rr: reference-row residual
    unsigned used = 0, seen = (lane == 0) ? 1u : 0u;
    int r = 0, j = 0, rej = 0, run = 0, iref = 0;
    bool converged = false;
    StopState st;
    st.floor2 = floor2;
    st.rtol2_m = rtol * rtol / (double)m;
    st.thr2 = thr * thr;
    st.fixed_rank = !(thr >= 0.0);
    const int limit = a.step_limit > 0 ? a.step_limit : kmax + n + 1;

    // reference row 0
    {
        const Pt<R> p0 = load_pt<R>(X, B.row0);
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int jj = lane + 32 * t;
            rr[t].init((jj < n) ? phi<KERN>(dist2(p0, load_pt<R>(X, B.col0 + jj)), c) : R(0));
        }
    }

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
            res[t].init(v);
        }
        for (int l0 = 0; l0 < r; l0 += 32) {
            const R vjc = (l0 + lane < r) ? V[(int64_t)(l0 + lane) * n + j] : R(0);
            const int lend = min(r - l0, 32);
            for (int l = 0; l < lend; l += WB) {
                R sv[WB], uv[WB][MAXR];
#pragma unroll
                for (int e = 0; e < WB; ++e) {
                    sv[e] = __shfl_sync(0xffffffffu, vjc, (l + e) & 31);
                    const R* Ul = U + (int64_t)(l0 + l + e) * m;
#pragma unroll
                    for (int t = 0; t < MAXR; ++t) {
                        const int i = lane + 32 * t;
                        uv[e][t] = (i < m && l + e < lend) ? Ul[i] : R(0);
                    }
                }
#pragma unroll
                for (int e = 0; e < WB; ++e)
#pragma unroll
                    for (int t = 0; t < MAXR; ++t) res[t].sub(uv[e][t], sv[e]);
            }
        }
        R best = -1;
        int bi = 0x7fffffff;
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            acc[t] = res[t].value();
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
            // or stop after rej_run rejections in a row
            ++rej;
            if (++run >= rej_run<R>()) {
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
        if ((bi & 31) == lane) seen |= 1u << (bi >> 5);
        R* __restrict__ Ur = U + (int64_t)r * m;
        R uiref = 0;
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int i = lane + 32 * t;
            if (i < m) {
                acc[t] = acc[t] / piv;
                Ur[i] = acc[t];
            }
            if (t == (iref >> 5)) uiref = acc[t];
        }
        uiref = __shfl_sync(0xffffffffu, uiref, iref & 31);
        // residual row v = A(i_r, :)^T - sum_{l<r} (u_l)_{i_r} v_l
        const Pt<R> pi = load_pt<R>(X, B.row0 + bi);
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int jj = lane + 32 * t;
            res[t].init((jj < n) ? phi<KERN>(dist2(pi, load_pt<R>(X, B.col0 + jj)), c) : R(0));
        }
        for (int l0 = 0; l0 < r; l0 += 32) {
            const R uic = (l0 + lane < r) ? U[(int64_t)(l0 + lane) * m + bi] : R(0);
            const int lend = min(r - l0, 32);
            for (int l = 0; l < lend; l += WB) {
                R su[WB], vv[WB][MAXR];
#pragma unroll
                for (int e = 0; e < WB; ++e) {
                    su[e] = __shfl_sync(0xffffffffu, uic, (l + e) & 31);
                    const R* Vl = V + (int64_t)(l0 + l + e) * n;
#pragma unroll
                    for (int t = 0; t < MAXR; ++t) {
                        const int jj = lane + 32 * t;
                        vv[e][t] = (jj < n && l + e < lend) ? Vl[jj] : R(0);
                    }
                }
#pragma unroll
                for (int e = 0; e < WB; ++e)
#pragma unroll
                    for (int t = 0; t < MAXR; ++t) res[t].sub(su[e], vv[e][t]);
            }
        }
        R* __restrict__ Vr = V + (int64_t)r * n;
        TSum<R> tu, tv;
        tu.init();
        tv.init();
        R rmax = 0;
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            vv[t] = res[t].value();
            const int i = lane + 32 * t;
            if (i < n) {
                Vr[i] = vv[t];
                tv.add(vv[t] * vv[t]);
                rr[t].sub(uiref, vv[t]);
                rmax = max(rmax, fabs(rr[t].value()));
            }
            if (i < m) tu.add(acc[t] * acc[t]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tu.shfl_join(o);
            tv.shfl_join(o);
        }
        rmax = warp_max(rmax);
        // cross terms (u_r . u_l)(v_l . v_r), reduced and summed in R
        // (LC ranks at a time, one reduce-scatter per side; the writer lane
        // of rank l0 + e keeps its products, the lanes' sums join at the end)
        TSum<R> tc;
        tc.init();
        for (int l0 = 0; l0 < r; l0 += LC) {
            R pu[LC], pv[LC];
#pragma unroll
            for (int e = 0; e < LC; ++e) {
                const R* Ul = U + (int64_t)(l0 + e) * m;
                const R* Vl = V + (int64_t)(l0 + e) * n;
                R du = 0, dv = 0;
#pragma unroll
                for (int t = 0; t < MAXR; ++t) {
                    const int i = lane + 32 * t;
                    const R ul = (i < m && l0 + e < r) ? Ul[i] : R(0);
                    const R vl = (i < n && l0 + e < r) ? Vl[i] : R(0);
                    du = fma(acc[t], ul, du);
                    dv = fma(vl, vv[t], dv);
                }
                pu[e] = du;
                pv[e] = dv;
            }
            const R su = warp_scatter(pu), sv = warp_scatter(pv);
            if (scatter_writer(lane) && l0 + scatter_elem(lane) < r) tc.add(su * sv);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tc.shfl_join(o);
        bool resolved, stop_ok;
        stop_step(st, tu, tv, tc.rvalue(), rmax, resolved, stop_ok);
        ++r;
        // a resolved reference row (max |residual| <= tol sqrt(S2 / m)) moves
        // to the lowest row not seen yet
        if (resolved) {
            int cand = 0x7fffffff;
#pragma unroll
            for (int t = 0; t < MAXR; ++t) {
                const int i = lane + 32 * t;
                if (i < m && !((seen >> t) & 1u)) {
                    cand = i;
                    break;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
            if (cand != 0x7fffffff) {
                iref = cand;
                if ((iref & 31) == lane) seen |= 1u << (iref >> 5);
                const Pt<R> pr = load_pt<R>(X, B.row0 + iref);
#pragma unroll
                for (int t = 0; t < MAXR; ++t) {
                    const int jj = lane + 32 * t;
                    res[t].init((jj < n) ? phi<KERN>(dist2(pr, load_pt<R>(X, B.col0 + jj)), c) : R(0));
                }
                for (int l0 = 0; l0 < r; l0 += 32) {
                    const R uic = (l0 + lane < r) ? U[(int64_t)(l0 + lane) * m + iref] : R(0);
                    const int lend = min(r - l0, 32);
                    for (int l = 0; l < lend; l += WB) {
                        R su[WB], vv[WB][MAXR];
#pragma unroll
                        for (int e = 0; e < WB; ++e) {
                            su[e] = __shfl_sync(0xffffffffu, uic, (l + e) & 31);
                            const R* Vl = V + (int64_t)(l0 + l + e) * n;
#pragma unroll
                            for (int t = 0; t < MAXR; ++t) {
                                const int jj = lane + 32 * t;
                                vv[e][t] = (jj < n && l + e < lend) ? Vl[jj] : R(0);
                            }
                        }
#pragma unroll
                        for (int e = 0; e < WB; ++e)
#pragma unroll
                            for (int t = 0; t < MAXR; ++t) res[t].sub(su[e], vv[e][t]);
                    }
                }
                rmax = 0;
#pragma unroll
                for (int t = 0; t < MAXR; ++t) {
                    rr[t] = res[t];
                    if (lane + 32 * t < n) rmax = max(rmax, fabs(rr[t].value()));
                }
                rmax = warp_max(rmax);
                resolved = ref_resolved(st, rmax);
            }
        }
        if (stop_ok && resolved) {
            converged = true;
            break;
        }
        if (r >= kmax) break;
        // next column: largest reference-row residual over unused columns
        R bv = -1;
        int bj = 0x7fffffff;
#pragma unroll
        for (int t = 0; t < MAXR; ++t) {
            const int jj = lane + 32 * t;
            if (jj < n && !((used >> t) & 1u) && fabs(rr[t].value()) > bv) {
                bv = fabs(rr[t].value());
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
// to all CS * CTA_NT threads, so every thread owns the same rows and columns
// in every pass. A reduction first combines inside each CTA, then every CTA
// reads the partials of all CTAs of its cluster from distributed shared
// memory in rank order, so all CTAs reach identical values and follow the
// same control flow. Partials are double-buffered, so one cluster barrier per
// reduction suffices. Used columns, seen rows and the reference-row residual
// live in global scratch owned by the cluster.
// --------------------------------------------------------------------------
// The reduced values of one step: sums, maxima, an argmax with its signed
// value (ties to the lowest index) and a minimum index. Each thread keeps one
// in its own type R (compensated sums, exact maxima); warps, CTAs and the
// cluster combine them in R, in a fixed order, and only the cluster result is
// widened to double (Red).
struct Red {
    double s0, s1;
    double x0, x1;
    double av, aval;
    int ai, mn;
};

template <class R>
struct LRed {
    TSum<R> s0, s1;
    R x0, x1, av, aval;
    int ai, mn;
    __device__ __forceinline__ void init()
    {
        s0.init();
        s1.init();
        x0 = x1 = R(0);
        av = R(-1);
        aval = R(0);
        ai = mn = 0x7fffffff;
    }
    __device__ __forceinline__ void join(const LRed& o)
    {
        s0.join(o.s0);
        s1.join(o.s1);
        x0 = max(x0, o.x0);
        x1 = max(x1, o.x1);
        if (o.av > av || (o.av == av && o.ai < ai)) {
            av = o.av;
            ai = o.ai;
            aval = o.aval;
        }
        mn = min(mn, o.mn);
    }
    // butterfly step: every lane ends with the same values
    __device__ __forceinline__ void shfl_join(int o)
    {
        s0.shfl_join(o);
        s1.shfl_join(o);
        x0 = max(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        const R oav = __shfl_xor_sync(0xffffffffu, av, o);
        const R oaval = __shfl_xor_sync(0xffffffffu, aval, o);
        const int oai = __shfl_xor_sync(0xffffffffu, ai, o);
        if (oav > av || (oav == av && oai < ai)) {
            av = oav;
            ai = oai;
            aval = oaval;
        }
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    __device__ __forceinline__ Red widen() const
    {
        Red t;
        t.s0 = s0.value();
        t.s1 = s1.value();
        t.x0 = (double)x0;
        t.x1 = (double)x1;
        t.av = (double)av;
        t.aval = (double)aval;
        t.ai = ai;
        t.mn = mn;
        return t;
    }
};

template <class R>
struct ClPart {
    LRed<R> q;
    double du[KBUF], dv[KBUF];
};

// Decisions of one step, taken once per CTA by the thread that forms the
// cluster result (every CTA of a cluster takes the same ones).
struct Ctl {
    double rlim2;    // tol^2 S2 / m: squared limit of a resolved reference row
    int resolved;    // reference-row residual within the limit
    int stop_ok;     // |u||v| <= thr sqrt(S2)
};

template <class R>
struct ClShared {
    ClPart<R> part[2];
    LRed<R> wq[CTA_WARPS];
    R wl[CTA_WARPS][KBUF];   // per-warp partial dots
    R wm[CTA_WARPS][KBUF];
    LRed<R> out;             // broadcast: the cluster-wide result
    Ctl ctl;
};

struct NoFin {
    __device__ __forceinline__ void operator()(const Red&, double) const {}
};

// Cluster-wide reduction of q (and, with ndots > 0, of the per-warp dot
// partials in sh.wl / sh.wm, whose cross sum is handed to fin); thread 0 of
// every CTA runs fin on the result widened to double, which may write
// sh.ctl; every thread of every CTA receives the result in R. No barrier is
// needed after the broadcast is read: the next reduction's first barrier
// orders those reads before sh.out and sh.ctl are written again.
template <class CL, class R, class FIN>
__device__ LRed<R> cl_reduce(CL& cl, ClShared<R>& sh, int& ph, const LRed<R>& lq, int ndots,
                             const FIN& fin)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int CS = (int)cl.num_blocks();
    LRed<R> q = lq;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q.shfl_join(o);
    if (lane == 0) sh.wq[w] = q;
    __syncthreads();
    ClPart<R>& P = sh.part[ph];
    if (tid == 0) {
        LRed<R> t = sh.wq[0];
        for (int k = 1; k < CTA_WARPS; ++k) t.join(sh.wq[k]);
        P.q = t;
    }
    if (tid < ndots) {
        TSum<R> su, sv;
        su.init();
        sv.init();
        for (int k = 0; k < CTA_WARPS; ++k) {
            su.add(sh.wl[k][tid]);
            sv.add(sh.wm[k][tid]);
        }
        P.du[tid] = su.value();
        P.dv[tid] = sv.value();
    }
    cl.sync();
    if (w == 0) {
        double cr = 0.0;
        for (int l0 = 0; l0 < ndots; l0 += 32) {
            const int l = l0 + lane;
            double su = 0.0, sv = 0.0;
            if (l < ndots)
                for (int k = 0; k < CS; ++k) {
                    const ClPart<R>* Q = cl.map_shared_rank(&sh.part[ph], k);
                    su += Q->du[l];
                    sv += Q->dv[l];
                }
            cr += warp_sum(su * sv);
        }
        if (lane == 0) {
            LRed<R> t = cl.map_shared_rank(&sh.part[ph], 0)->q;
            for (int k = 1; k < CS; ++k) t.join(cl.map_shared_rank(&sh.part[ph], k)->q);
            fin(t.widen(), cr);
            sh.out = t;
        }
    }
    ph ^= 1;
    __syncthreads();
    return sh.out;
}

template <class R, int KERN>
__global__ void __launch_bounds__(CTA_NT, 3)
k_aca_cluster(KernelParams kp, DeviceCoords X, AcaArgs a, const uint32_t* __restrict__ order,
              int64_t nblocks, double thr, uint32_t* __restrict__ usedpool,
              uint32_t* __restrict__ seenpool, R* __restrict__ rrpool, int64_t words,
              int64_t maxdim)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks();
    const int crank = (int)cl.block_rank();
    __shared__ R sg[KBUF];
    __shared__ ClShared<R> sh;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int gt = crank * CTA_NT + tid, GT = CS * CTA_NT;
    const int64_t cid = blockIdx.x / CS, ncl = gridDim.x / CS;
    uint32_t* used = usedpool + cid * words;
    uint32_t* seen = seenpool + cid * words;
    R* rr = rrpool + cid * maxdim;   // reference-row residual
    const R c = kconst<R>(kp);
    const R eps0 = (R)a.eps0;
    const double rtol = a.eps > 0.0 ? a.eps : a.eps0;
    const double thr2 = thr * thr;
    const NoFin nofin;
    int ph = 0;

    for (int64_t q = cid; q < nblocks; q += ncl) {
        const uint32_t b = order[q];
        const Blk B = a.blk[b];
        const int m = B.m, n = B.n;
        const int kres = a.kres[b];
        const int kmax = min(kres, min(m, n));
        R* __restrict__ U = reinterpret_cast<R*>(a.Uptr[b]);
        R* __restrict__ V = reinterpret_cast<R*>(a.Vptr[b]);
        const int wn = (n + 31) / 32, wm = (m + 31) / 32;
        // ||S_r||_F^2, the floor and tol^2 / m: kept and used by thread 0 of
        // each CTA only (the other threads do no double arithmetic)
        double S2 = 0.0, floor2 = 0.0, rtol2_m = 0.0;
        if (tid == 0) {
            floor2 = a.bset ? (double)m * (double)n / (double)a.set_n[a.bset[b]] : 0.0;
            rtol2_m = rtol * rtol / (double)m;
        }
        // the step's decisions from the row reduction: S2, the reference-row
        // limit and both tests in squared form
        auto fin_row = [&](const Red& o, double cross) {
            S2 += 2.0 * cross + o.s0 * o.s1;
            const double S2f = fmax(S2, floor2);
            const double rlim2 = rtol2_m * S2f;
            sh.ctl.rlim2 = rlim2;
            sh.ctl.resolved = !(o.x1 * o.x1 > rlim2);
            sh.ctl.stop_ok = thr >= 0.0 && o.s0 * o.s1 <= thr2 * S2f;
        };
        auto fin_ref = [&](const Red& o, double) {
            sh.ctl.resolved = !(o.x1 * o.x1 > sh.ctl.rlim2);
        };
        for (int k = gt; k < wn; k += GT) used[k] = 0u;
        for (int k = gt; k < wm; k += GT) seen[k] = 0u;
        cl.sync();
        if (gt == 0) seen[0] = 1u;
        // reference row 0
        {
            const Pt<R> p0 = load_pt<R>(X, B.row0);
            for (int jj = gt; jj < n; jj += GT) {
                rr[jj] = phi<KERN>(dist2(p0, load_pt<R>(X, B.col0 + jj)), c);
            }
        }
        int r = 0, j = 0, rej = 0, run = 0, iref = 0;
        bool converged = false;
        const int limit = a.step_limit > 0 ? a.step_limit : kmax + n + 1;
        for (int it = 0; r < kmax; ++it) {
            if (it > limit) {
                if (gt == 0) atomicOr(a.status, 1);
                break;
            }
            if (gt == 0) used[j >> 5] |= 1u << (j & 31);
            if (tid < r) sg[tid] = V[(int64_t)tid * n + j];
            __syncthreads();
            // residual column, its pivot and u^ at the reference row
            const Pt<R> pj = load_pt<R>(X, B.col0 + j);
            R* __restrict__ Ur = U + (int64_t)r * m;
            LRed<R> qc;
            qc.init();
            // rows in chunks of UNR per thread so that UNR loads are in flight
            for (int i0 = gt; i0 < m; i0 += UNR * GT) {
                Resid<R> rs_[UNR];
#pragma unroll
                for (int q = 0; q < UNR; ++q) {
                    const int i = i0 + q * GT;
                    R a0 = 0;
                    if (i < m) {
                        a0 = phi<KERN>(dist2(load_pt<R>(X, B.row0 + i), pj), c);
                        qc.x0 = max(qc.x0, fabs(a0));
                    }
                    rs_[q].init(a0);
                }
                for (int l = 0; l < r; ++l) {
                    const R vl = sg[l];
                    const R* Ul = U + (int64_t)l * m;
                    R uv[UNR];
#pragma unroll
                    for (int q = 0; q < UNR; ++q) uv[q] = (i0 + q * GT < m) ? Ul[i0 + q * GT] : R(0);
#pragma unroll
                    for (int q = 0; q < UNR; ++q) rs_[q].sub(uv[q], vl);
                }
#pragma unroll
                for (int q = 0; q < UNR; ++q) {
                    const int i = i0 + q * GT;
                    if (i >= m) continue;
                    const R v = rs_[q].value();
                    Ur[i] = v;
                    if (fabs(v) > qc.av) {
                        qc.av = fabs(v);
                        qc.ai = i;
                        qc.aval = v;
                    }
                    if (i == iref) qc.s0.set(v);
                }
            }
            const LRed<R> oc = cl_reduce(cl, sh, ph, qc, 0, nofin);
            const R best = oc.av, amax = oc.x0;
            const int bi = oc.ai;
            if (!(best > eps0 * amax)) {
                ++rej;
                if (++run >= rej_run<R>()) {
                    converged = true;
                    break;
                }
                // lowest unused column over the whole cluster
                LRed<R> qn;
                qn.init();
                for (int k = gt; k < wn; k += GT) {
                    uint32_t free_bits = ~used[k];
                    if (k == wn - 1 && (n & 31)) free_bits &= (1u << (n & 31)) - 1u;
                    if (free_bits) {
                        qn.mn = k * 32 + __ffs(free_bits) - 1;
                        break;
                    }
                }
                const int cand = cl_reduce(cl, sh, ph, qn, 0, nofin).mn;
                if (cand == 0x7fffffff || cand >= n) {
                    converged = true;
                    break;
                }
                j = cand;
                continue;
            }
            run = 0;
            const R piv = oc.aval;
            const R uiref = oc.s0.s / piv;
            if (gt == 0) seen[bi >> 5] |= 1u << (bi & 31);
            if (tid < r) sg[tid] = U[(int64_t)tid * m + bi];
            __syncthreads();
            // residual row, scaled column, reference row, norms, next column
            const Pt<R> pi = load_pt<R>(X, B.row0 + bi);
            R* __restrict__ Vr = V + (int64_t)r * n;
            LRed<R> qr;
            qr.init();
            for (int j0 = gt; j0 < n; j0 += UNR * GT) {
                Resid<R> rs_[UNR];
#pragma unroll
                for (int q = 0; q < UNR; ++q) {
                    const int jj = j0 + q * GT;
                    rs_[q].init(jj < n ? phi<KERN>(dist2(pi, load_pt<R>(X, B.col0 + jj)), c) : R(0));
                }
                for (int l = 0; l < r; ++l) {
                    const R ul = sg[l];
                    const R* Vl = V + (int64_t)l * n;
                    R vv[UNR];
#pragma unroll
                    for (int q = 0; q < UNR; ++q) vv[q] = (j0 + q * GT < n) ? Vl[j0 + q * GT] : R(0);
#pragma unroll
                    for (int q = 0; q < UNR; ++q) rs_[q].sub(ul, vv[q]);
                }
#pragma unroll
                for (int q = 0; q < UNR; ++q) {
                    const int jj = j0 + q * GT;
                    if (jj >= n) continue;
                    const R v = rs_[q].value();
                    Vr[jj] = v;
                    qr.s1.add(v * v);
                    Resid<R> rx;
                    rx.init(rr[jj]);
                    rx.sub(uiref, v);
                    const R x = rx.value();
                    rr[jj] = x;
                    qr.x1 = max(qr.x1, fabs(x));
                    if (!((used[jj >> 5] >> (jj & 31)) & 1u) && fabs(x) > qr.av) {
                        qr.av = fabs(x);
                        qr.ai = jj;
                    }
                }
            }
#pragma unroll 4
            for (int i = gt; i < m; i += GT) {
                const R u = Ur[i] / piv;
                Ur[i] = u;
                qr.s0.add(u * u);
            }
            for (int l = 0; l < r; ++l) {
                const R* Ul = U + (int64_t)l * m;
                const R* Vl = V + (int64_t)l * n;
                R du = 0, dv = 0;
                for (int i0 = gt; i0 < m; i0 += UNR * GT) {
                    R a[UNR], b[UNR];
#pragma unroll
                    for (int q = 0; q < UNR; ++q) {
                        const int i = i0 + q * GT;
                        a[q] = i < m ? Ur[i] : R(0);
                        b[q] = i < m ? Ul[i] : R(0);
                    }
#pragma unroll
                    for (int q = 0; q < UNR; ++q) du += a[q] * b[q];
                }
                for (int j0 = gt; j0 < n; j0 += UNR * GT) {
                    R a[UNR], b[UNR];
#pragma unroll
                    for (int q = 0; q < UNR; ++q) {
                        const int jj = j0 + q * GT;
                        a[q] = jj < n ? Vl[jj] : R(0);
                        b[q] = jj < n ? Vr[jj] : R(0);
                    }
#pragma unroll
                    for (int q = 0; q < UNR; ++q) dv += a[q] * b[q];
                }
                const R ddu = warp_sum(du), ddv = warp_sum(dv);
                if (lane == 0) {
                    sh.wl[w][l] = ddu;
                    sh.wm[w][l] = ddv;
                }
            }
            const LRed<R> orr = cl_reduce(cl, sh, ph, qr, r, fin_row);
            int nj = orr.ai;
            ++r;
            bool resolved = sh.ctl.resolved;
            const bool stop_ok = sh.ctl.stop_ok;
            // a resolved reference row moves to the lowest row not seen yet
            if (resolved) {
                LRed<R> qs;
                qs.init();
                for (int k = gt; k < wm; k += GT) {
                    uint32_t free_bits = ~seen[k];
                    if (k == wm - 1 && (m & 31)) free_bits &= (1u << (m & 31)) - 1u;
                    if (free_bits) {
                        qs.mn = k * 32 + __ffs(free_bits) - 1;
                        break;
                    }
                }
                const int cand = cl_reduce(cl, sh, ph, qs, 0, nofin).mn;
                if (cand != 0x7fffffff && cand < m) {
                    iref = cand;
                    if (gt == 0) seen[iref >> 5] |= 1u << (iref & 31);
                    if (tid < r) sg[tid] = U[(int64_t)tid * m + iref];
                    __syncthreads();
                    const Pt<R> pr = load_pt<R>(X, B.row0 + iref);
                    LRed<R> qf;
                    qf.init();
                    for (int j0 = gt; j0 < n; j0 += UNR * GT) {
                        Resid<R> rs_[UNR];
#pragma unroll
                        for (int q = 0; q < UNR; ++q) {
                            const int jj = j0 + q * GT;
                            rs_[q].init(jj < n ? phi<KERN>(dist2(pr, load_pt<R>(X, B.col0 + jj)), c) : R(0));
                        }
                        for (int l = 0; l < r; ++l) {
                            const R ul = sg[l];
                            const R* Vl = V + (int64_t)l * n;
                            R vv[UNR];
#pragma unroll
                            for (int q = 0; q < UNR; ++q) vv[q] = (j0 + q * GT < n) ? Vl[j0 + q * GT] : R(0);
#pragma unroll
                            for (int q = 0; q < UNR; ++q) rs_[q].sub(ul, vv[q]);
                        }
#pragma unroll
                        for (int q = 0; q < UNR; ++q) {
                            const int jj = j0 + q * GT;
                            if (jj >= n) continue;
                            const R x = rs_[q].value();
                            rr[jj] = x;
                            qf.x1 = max(qf.x1, fabs(x));
                            if (!((used[jj >> 5] >> (jj & 31)) & 1u) && fabs(x) > qf.av) {
                                qf.av = fabs(x);
                                qf.ai = jj;
                            }
                        }
                    }
                    const LRed<R> of = cl_reduce(cl, sh, ph, qf, 0, fin_ref);
                    resolved = sh.ctl.resolved;
                    nj = of.ai;
                }
            }
            if (stop_ok && resolved) {
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

// --------------------------------------------------------------------------
// Blocks with 512 < max(m, n) <= 65536: one CTA or one thread-block cluster
// of CS CTAs per block, persistent over the blocks of a size class. Thread g
// of the cluster (g = rank * NT + tid, G = CS * NT) owns the rows g + qG and
// the columns g + qG, q < R, and keeps in registers the residual column at
// its rows, the reference-row residual at its columns and bit masks of its
// used columns and seen rows, so a step touches global memory only for the
// block's earlier factor columns, and loads LC ranks of R rows at once.
//
// The cross terms of ||S_r||_F^2 come out of the same passes. The column
// pass subtracts the ranks in batches [l0, l0 + LC); before batch l0 the
// residual is w = A(:, j) - sum_{l' < l0} u_l' (v_l')_j, and for l in the
// batch
//     u^ . u_l = w . u_l - sum_{l' >= l0} (u_l' . u_l) (v_l')_j,
// so the pass accumulates w . u_l beside the residual, and the Gram matrix
// of u_0 .. u_{r-1} (shared memory) corrects the sums afterwards; likewise on
// the row side with the Gram matrix of the v's. A step therefore has two
// reductions (three when the reference row moves).
// --------------------------------------------------------------------------
constexpr int KG = 64;                       // largest rank of k_aca_big
constexpr int KGP = KG * (KG + 1) / 2;       // packed lower triangle

__device__ __forceinline__ int pk(int a, int b)   // a >= b
{
    return a * (a + 1) / 2 + b;
}

// Values reduced over the threads of a cluster in one step.
template <class T>
struct BRed {
    TSum<T> s0, s1;   // sums
    T x0;             // maximum
    T av, aval;       // argmax: |value|, signed value
    int ai;           // argmax index (ties: lowest index)
    int mn;           // minimum index
    T pick;           // a value contributed by a single thread (others 0)
    __device__ __forceinline__ void init()
    {
        s0.init();
        s1.init();
        x0 = T(0);
        av = T(-1);
        aval = T(0);
        ai = mn = 0x7fffffff;
        pick = T(0);
    }
    __device__ __forceinline__ void take(T oav, T oaval, int oai)
    {
        if (oav > av || (oav == av && oai < ai)) {
            av = oav;
            ai = oai;
            aval = oaval;
        }
    }
    __device__ __forceinline__ void join(const BRed& o)
    {
        s0.join(o.s0);
        s1.join(o.s1);
        x0 = max(x0, o.x0);
        take(o.av, o.aval, o.ai);
        mn = min(mn, o.mn);
        pick += o.pick;
    }
    __device__ __forceinline__ void shfl_join(int o)
    {
        s0.shfl_join(o);
        s1.shfl_join(o);
        x0 = max(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        const T oav = __shfl_xor_sync(0xffffffffu, av, o);
        const T oaval = __shfl_xor_sync(0xffffffffu, aval, o);
        const int oai = __shfl_xor_sync(0xffffffffu, ai, o);
        take(oav, oaval, oai);
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        pick += __shfl_xor_sync(0xffffffffu, pick, o);
    }
    __device__ __forceinline__ void bcast(int src)
    {
        s0.s = __shfl_sync(0xffffffffu, s0.s, src);
        s1.s = __shfl_sync(0xffffffffu, s1.s, src);
        if constexpr (sizeof(TSum<T>) > sizeof(T)) {
            s0.c = __shfl_sync(0xffffffffu, s0.c, src);
            s1.c = __shfl_sync(0xffffffffu, s1.c, src);
        }
        x0 = __shfl_sync(0xffffffffu, x0, src);
        av = __shfl_sync(0xffffffffu, av, src);
        aval = __shfl_sync(0xffffffffu, aval, src);
        ai = __shfl_sync(0xffffffffu, ai, src);
        mn = __shfl_sync(0xffffffffu, mn, src);
        pick = __shfl_sync(0xffffffffu, pick, src);
    }
};

template <class T, int NW>
struct BigShared {
    T Gu[KGP], Gv[KGP];          // Gram matrices of the u's and of the v's
    T sgv[KG], sgu[KG];          // (v_l)_j and (u_l)_{i*} of the current step
    T wvec[NW][KG];              // per-warp partial dot products
    BRed<T> wq[NW];
    struct Part {
        BRed<T> q;
        T vec[KG];
    } part[2];                   // per-CTA partials, read by the whole cluster
    int resolved, stop_ok;       // decisions of thread 0
};


// Cluster-wide reduction of q and of the first nvec entries of the per-warp
// vectors sh.wvec. Every thread receives the scalar result; lane L of every
// warp receives the vector entries L and L + 32 in vout. Partials are double
// buffered (ph), so two barriers per reduction suffice: a later reduction
// writes the other buffer, and the one after that only once every CTA has
// passed the cluster barrier in between.
template <class T, int NT, class CL>
__device__ __noinline__ BRed<T> big_reduce(CL& cl, int CS, BigShared<T, NT / 32>& sh, int& ph,
                                           BRed<T> q, int nvec, T (&vout)[KG / 32])
{
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q.shfl_join(o);
    if (lane == 0) sh.wq[w] = q;
    __syncthreads();
    auto& P = sh.part[ph];
    if (tid == 0) {
        BRed<T> t = sh.wq[0];
        for (int k = 1; k < NW; ++k) t.join(sh.wq[k]);
        P.q = t;
    }
    for (int l = tid; l < nvec; l += NT) {
        T s = T(0);
        for (int k = 0; k < NW; ++k) s += sh.wvec[k][l];
        P.vec[l] = s;
    }
    cl.sync();
    BRed<T> t;
    if (CS == 1) {
        t = P.q;
    } else {
        if (lane < CS) t = cl.map_shared_rank(&sh.part[ph], lane)->q;
        else t.init();
        for (int o = 1; o < CS; o <<= 1) t.shfl_join(o);
        t.bcast(0);
    }
#pragma unroll
    for (int s = 0; s < KG / 32; ++s) {
        const int l = lane + 32 * s;
        T v = T(0);
        if (l < nvec)
            for (int k = 0; k < CS; ++k) v += cl.map_shared_rank(&sh.part[ph], k)->vec[l];
        vout[s] = v;
    }
    ph ^= 1;
    return t;
}

template <class T, int KERN, int R, int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
k_aca_big(KernelParams kp, DeviceCoords X, AcaArgs a, const uint32_t* __restrict__ order,
          int64_t nblocks, double thr)
{
    namespace cg = cooperative_groups;
    constexpr int NW = NT / 32;
    static_assert(R <= 32, "bit masks hold 32 rows per thread");
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks();
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int g = (int)cl.block_rank() * NT + tid, G = CS * NT;
    const int64_t cid = blockIdx.x / CS, ncl = gridDim.x / CS;
    __shared__ BigShared<T, NW> sh;
    const T c = kconst<T>(kp);
    const T eps0 = (T)a.eps0;
    const double rtol = a.eps > 0.0 ? a.eps : a.eps0;
    const double thr2 = thr * thr;
    int ph = 0;

    for (int64_t qb = cid; qb < nblocks; qb += ncl) {
        const uint32_t b = order[qb];
        const Blk B = a.blk[b];
        const int m = B.m, n = B.n;
        const int kres = a.kres[b];
        const int kmax = min(min(kres, KG), min(m, n));
        if (max(m, n) > R * G) {   // the host routes no such block here
            if (g == 0) atomicOr(a.status, 2);
            continue;
        }
        T* __restrict__ U = reinterpret_cast<T*>(a.Uptr[b]);
        T* __restrict__ V = reinterpret_cast<T*>(a.Vptr[b]);
        // ||S_r||_F^2 and the limits of the tests: thread 0 of each CTA only
        StopState st;
        if (tid == 0) {
            st.floor2 = a.bset ? (double)m * (double)n / (double)a.set_n[a.bset[b]] : 0.0;
            st.rtol2_m = rtol * rtol / (double)m;
            st.thr2 = thr2;
            st.fixed_rank = !(thr >= 0.0);
        }
        T uh[R], rr[R];
        unsigned used = 0u, seen = (g == 0) ? 1u : 0u;
        {
            const Pt<T> p0 = load_pt<T>(X, B.row0);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int jj = g + q * G;
                rr[q] = jj < n ? phi<KERN>(dist2(p0, load_pt<T>(X, B.col0 + jj)), c) : T(0);
            }
        }
        int r = 0, j = 0, rej = 0, run = 0, iref = 0;
        bool converged = false;
        const int limit = a.step_limit > 0 ? a.step_limit : kmax + n + 1;
        T du[KG / 32];
        for (int it = 0; r < kmax; ++it) {
            if (it > limit) {
                if (g == 0) atomicOr(a.status, 1);
                break;
            }
            if (j % G == g) used |= 1u << (j / G);
            if (w == 0)
                for (int l = lane; l < r; l += 32) sh.sgv[l] = __ldcg(V + (int64_t)l * n + j);
            // ---- column pass: u^ = a - sum_l u_l (v_l)_j and a . u_l
            BRed<T> qc;
            qc.init();
            {
                const Pt<T> pj = load_pt<T>(X, B.col0 + j);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int i = g + q * G;
                    T v = T(0);
                    if (i < m) v = phi<KERN>(dist2(load_pt<T>(X, B.row0 + i), pj), c);
                    qc.x0 = max(qc.x0, fabs(v));
                    uh[q] = v;
                }
            }
            for (int l0 = 0; l0 < r; l0 += LC) {
                T sv[LC], p[LC];
#pragma unroll
                for (int e = 0; e < LC; ++e) {
                    sv[e] = (l0 + e < r) ? __ldcg(V + (int64_t)(l0 + e) * n + j) : T(0);
                    p[e] = T(0);
                }
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int i = g + q * G;
                    T u[LC];
#pragma unroll
                    for (int e = 0; e < LC; ++e)
                        u[e] = (i < m && l0 + e < r) ? __ldcg(U + (int64_t)(l0 + e) * m + i) : T(0);
#pragma unroll
                    for (int e = 0; e < LC; ++e) p[e] = fma(uh[q], u[e], p[e]);
#pragma unroll
                    for (int e = 0; e < LC; ++e) uh[q] = fma(-u[e], sv[e], uh[q]);
                }
                const T ps = warp_scatter(p);
                const int e = scatter_elem(lane);
                if (scatter_writer(lane) && l0 + e < r) sh.wvec[w][l0 + e] = ps;
            }
            bool have_mn = false;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = g + q * G;
                if (i < m) {
                    qc.take(fabs(uh[q]), uh[q], i);
                    if (i == iref) qc.pick = uh[q];
                }
                const int jj = g + q * G;
                if (!have_mn && jj < n && !((used >> q) & 1u)) {
                    qc.mn = jj;
                    have_mn = true;
                }
            }
            T Pv[KG / 32];
            const BRed<T> oc = big_reduce<T, NT>(cl, CS, sh, ph, qc, r, Pv);
            if (!(oc.av > eps0 * oc.x0)) {
                // column already represented: take the lowest unused column,
                // or stop after rej_run rejections in a row
                ++rej;
                if (++run >= rej_run<T>() || oc.mn >= n) {
                    converged = true;
                    break;
                }
                j = oc.mn;
                continue;
            }
            run = 0;
            const T piv = oc.aval;
            const int bi = oc.ai;
            const T uiref = oc.pick / piv;
            if (bi % G == g) seen |= 1u << (bi / G);
            // u_r . u_l = (a . u_l - sum_l' Gu(l, l') (v_l')_j) / piv
#pragma unroll
            for (int s = 0; s < KG / 32; ++s) {
                const int l = lane + 32 * s;
                T x = T(0);
                if (l < r) {
                    x = Pv[s];
                    for (int l2 = l - l % LC; l2 < r; ++l2)
                        x = fma(-sh.Gu[l >= l2 ? pk(l, l2) : pk(l2, l)], sh.sgv[l2], x);
                    x = x / piv;
                }
                du[s] = x;
            }
            if (w == 0)
                for (int l = lane; l < r; l += 32) sh.sgu[l] = __ldcg(U + (int64_t)l * m + bi);
            // ---- u_r = u^ / piv, then the row pass: v = A(i*, :) - sum_l (u_l)_i* v_l
            BRed<T> qr;
            qr.init();
            T* __restrict__ Ur = U + (int64_t)r * m;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = g + q * G;
                if (i < m) {
                    const T u = uh[q] / piv;
                    Ur[i] = u;
                    qr.s0.add(u * u);
                }
            }
            {
                const Pt<T> pi = load_pt<T>(X, B.row0 + bi);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int jj = g + q * G;
                    uh[q] = jj < n ? phi<KERN>(dist2(pi, load_pt<T>(X, B.col0 + jj)), c) : T(0);
                }
            }
            for (int l0 = 0; l0 < r; l0 += LC) {
                T su[LC], p[LC];
#pragma unroll
                for (int e = 0; e < LC; ++e) {
                    su[e] = (l0 + e < r) ? __ldcg(U + (int64_t)(l0 + e) * m + bi) : T(0);
                    p[e] = T(0);
                }
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int jj = g + q * G;
                    T v[LC];
#pragma unroll
                    for (int e = 0; e < LC; ++e)
                        v[e] = (jj < n && l0 + e < r) ? __ldcg(V + (int64_t)(l0 + e) * n + jj) : T(0);
#pragma unroll
                    for (int e = 0; e < LC; ++e) p[e] = fma(uh[q], v[e], p[e]);
#pragma unroll
                    for (int e = 0; e < LC; ++e) uh[q] = fma(-su[e], v[e], uh[q]);
                }
                const T ps = warp_scatter(p);
                const int e = scatter_elem(lane);
                if (scatter_writer(lane) && l0 + e < r) sh.wvec[w][l0 + e] = ps;
            }
            T* __restrict__ Vr = V + (int64_t)r * n;
            bool have_mn2 = false;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int jj = g + q * G;
                if (jj < n) {
                    const T v = uh[q];
                    Vr[jj] = v;
                    qr.s1.add(v * v);
                    rr[q] = fma(-uiref, v, rr[q]);
                    const T x = fabs(rr[q]);
                    qr.x0 = max(qr.x0, x);
                    if (!((used >> q) & 1u)) qr.take(x, rr[q], jj);
                }
                const int i = g + q * G;
                if (!have_mn2 && i < m && !((seen >> q) & 1u)) {
                    qr.mn = i;
                    have_mn2 = true;
                }
            }
            T Qv[KG / 32];
            const BRed<T> orr = big_reduce<T, NT>(cl, CS, sh, ph, qr, r, Qv);
            // v_l . v_r = a' . v_l - sum_l' Gv(l, l') (u_l')_i*; cross terms of S2
            T cr = T(0), dv[KG / 32];
#pragma unroll
            for (int s = 0; s < KG / 32; ++s) {
                const int l = lane + 32 * s;
                T x = T(0);
                if (l < r) {
                    x = Qv[s];
                    for (int l2 = l - l % LC; l2 < r; ++l2)
                        x = fma(-sh.Gv[l >= l2 ? pk(l, l2) : pk(l2, l)], sh.sgu[l2], x);
                }
                dv[s] = x;
                cr = fma(du[s], x, cr);
            }
            if (w == 0) {
                cr = warp_sum(cr);
#pragma unroll
                for (int s = 0; s < KG / 32; ++s) {
                    const int l = lane + 32 * s;
                    if (l < r) {
                        sh.Gu[pk(r, l)] = du[s];
                        sh.Gv[pk(r, l)] = dv[s];
                    }
                }
                if (lane == 0) {
                    sh.Gu[pk(r, r)] = orr.s0.rvalue();
                    sh.Gv[pk(r, r)] = orr.s1.rvalue();
                    bool res, stp;
                    stop_step(st, orr.s0, orr.s1, cr, orr.x0, res, stp);
                    sh.resolved = res;
                    sh.stop_ok = stp;
                }
            }
            __syncthreads();
            ++r;
            bool resolved = sh.resolved;
            const bool stop_ok = sh.stop_ok;
            int nj = orr.ai;
            // a resolved reference row moves to the lowest row not seen yet
            if (resolved && orr.mn < m) {
                iref = orr.mn;
                if (iref % G == g) seen |= 1u << (iref / G);
                const Pt<T> pr = load_pt<T>(X, B.row0 + iref);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int jj = g + q * G;
                    uh[q] = jj < n ? phi<KERN>(dist2(pr, load_pt<T>(X, B.col0 + jj)), c) : T(0);
                }
                for (int l0 = 0; l0 < r; l0 += LC) {
                    T su[LC];
#pragma unroll
                    for (int e = 0; e < LC; ++e)
                        su[e] = (l0 + e < r) ? __ldcg(U + (int64_t)(l0 + e) * m + iref) : T(0);
#pragma unroll
                    for (int q = 0; q < R; ++q) {
                        const int jj = g + q * G;
                        T v[LC];
#pragma unroll
                        for (int e = 0; e < LC; ++e)
                            v[e] = (jj < n && l0 + e < r) ? __ldcg(V + (int64_t)(l0 + e) * n + jj) : T(0);
#pragma unroll
                        for (int e = 0; e < LC; ++e) uh[q] = fma(-su[e], v[e], uh[q]);
                    }
                }
                BRed<T> qf;
                qf.init();
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const int jj = g + q * G;
                    if (jj < n) {
                        rr[q] = uh[q];
                        const T x = fabs(rr[q]);
                        qf.x0 = max(qf.x0, x);
                        if (!((used >> q) & 1u)) qf.take(x, rr[q], jj);
                    }
                }
                T dummy[KG / 32];
                const BRed<T> of = big_reduce<T, NT>(cl, CS, sh, ph, qf, 0, dummy);
                if (tid == 0) sh.resolved = ref_resolved(st, of.x0);
                __syncthreads();
                resolved = sh.resolved;
                nj = of.ai;
            }
            if (stop_ok && resolved) {
                converged = true;
                break;
            }
            if (r >= kmax) break;
            if (nj >= n) {
                converged = true;
                break;
            }
            j = nj;
        }
        if (g == 0) {
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
void launch_cluster(const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                    const uint32_t* order, int64_t n, int cs, int64_t dim, double thr,
                    cudaStream_t s)
{
    int occ = 0;
    HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_aca_cluster<R, KERN>, CTA_NT, 0));
    int64_t nclusters = std::min<int64_t>(n, std::max<int64_t>(1, (int64_t)std::max(occ, 1) *
                                                                     num_sms() / cs));
    const int64_t words = ceil_div(dim, 32);
    DevBuf<uint32_t> usedpool((size_t)(nclusters * words), s);
    DevBuf<uint32_t> seenpool((size_t)(nclusters * words), s);
    DevBuf<R> rrpool((size_t)(nclusters * dim), s);
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
    HM_CUDA(cudaLaunchKernelEx(&cfg, k_aca_cluster<R, KERN>, kp, X, a, order, n, thr, usedpool.p,
                               seenpool.p, rrpool.p, words, dim));
    note_launch();
}

// One CTA (cs = 1) or one cluster of cs CTAs per block, as many as fit at once.
template <class R, int KERN, int RR, int NT>
void launch_big(const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                const uint32_t* order, int64_t n, int cs, double thr, cudaStream_t s)
{
    auto kern = k_aca_big<R, KERN, RR, NT>;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int64_t fit = 0;
    if (cs == 1) {
        int occ = 0;
        HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, 0));
        fit = (int64_t)std::max(occ, 1) * num_sms();
    } else {
        cfg.gridDim = dim3((unsigned)cs);
        int ncl = 0;
        HM_CUDA(cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg));
        fit = std::max(ncl, 1);
    }
    const int64_t nclusters = std::min<int64_t>(n, fit);
    cfg.gridDim = dim3((unsigned)(nclusters * cs));
    HM_CUDA(cudaLaunchKernelEx(&cfg, kern, kp, X, a, order, n, thr));
    note_launch();
}

template <class R, int KERN>
void launch_all(const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                const uint32_t* order, int64_t n, int cls, int64_t max_n, cudaStream_t s)
{
    const double thr = (a.eps > 0.0) ? a.eps * (1.0 - a.aca_eta) / (1.0 + a.eps) : -1.0;
    const unsigned wgrid = (unsigned)ceil_div(n * 32, WARP_NT);
    const int64_t dim = std::min<int64_t>(cls == ACA_NCLASS - 1 ? max_n : aca_class_dim(cls), max_n);
    if (cls >= 4 && cls < ACA_NCLASS - 1 && a.k_cap > KG) {
        // ranks above the Gram matrices' size: residuals in global scratch
        launch_cluster<R, KERN>(kp, X, a, order, n, dim <= 4096 ? 1 : dim <= 32768 ? 4 : 8, dim,
                                thr, s);
        HM_LAUNCH("aca");
        return;
    }
    switch (cls) {
    case 0: k_aca_warp<R, KERN, 2><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr); note_launch(); break;
    case 1: k_aca_warp<R, KERN, 4><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr); note_launch(); break;
    case 2: k_aca_warp<R, KERN, 8><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr); note_launch(); break;
    case 3: k_aca_warp<R, KERN, 16><<<wgrid, WARP_NT, 0, s>>>(kp, X, a, order, n, thr); note_launch(); break;
    case 4: launch_big<R, KERN, 8, 128>(kp, X, a, order, n, 1, thr, s); break;     // <= 1024
    case 5: launch_big<R, KERN, 8, 256>(kp, X, a, order, n, 1, thr, s); break;     // <= 2048
    case 6: launch_big<R, KERN, 8, 512>(kp, X, a, order, n, 1, thr, s); break;     // <= 4096
    case 7: launch_big<R, KERN, 8, 512>(kp, X, a, order, n, 2, thr, s); break;     // <= 8192
    case 8: launch_big<R, KERN, 8, 512>(kp, X, a, order, n, 4, thr, s); break;     // <= 16384
    case 9: launch_big<R, KERN, 8, 512>(kp, X, a, order, n, 8, thr, s); break;     // <= 32768
    case 10: launch_big<R, KERN, 16, 512>(kp, X, a, order, n, 8, thr, s); break;   // <= 65536
    default: launch_cluster<R, KERN>(kp, X, a, order, n, 8, dim, thr, s); break;
    }
    HM_LAUNCH("aca");
}

}  // namespace

}  // namespace hm
