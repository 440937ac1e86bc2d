// hm_aca_team.cuh -- batched ACA (Alg. 2, Sec. 5.4.1) by teams of W warps.
//
// One team of W warps (W = 1, 2, 4, 8, 16 or 32) compresses one admissible
// block at a time; a CTA holds max(4, W) warps, i.e. 4 / W teams when W < 4.
// Team thread g (g < G = 32 W) owns the rows g + q G and the columns g + q G
// (q < R) of its block and keeps in registers the residual column (or row)
// at those entries and the reference-row residual at its columns, so one
// team covers blocks with max(m, n) <= R G. The reductions of a step are
// warp butterflies, joined across the team's warps through shared memory
// (one named barrier per reduction); there is no CTA-wide or cluster-wide
// barrier, so a team never waits for another block.
//
// The readings of Alg. 2 are those of the other ACA kernels (hm_aca_impl.cuh):
// first column 0, row pivot argmax |u^| (lowest index on ties), rejection of
// a column whose residual is <= eps0 max |A(:, j)| (the lowest unused column
// is tried next; rej_run rejections in a row end the block), the next column
// is the argmax over unused columns of the reference row's residual, the
// reference row moves to the lowest row not yet seen once it is resolved,
// ||S_r||_F^2 by the textbook update with its cross terms, and the stopping
// rule |u_r||v_r| <= thr ||S_r||_F with the reference row resolved. The cross
// terms come out of the residual passes with Gram-matrix corrections (the
// identity in the comment of k_aca_big); the Gram matrices of the u's and
// the v's live in shared memory, packed, for ranks up to KT, a launch
// parameter (16, 32 or 64) chosen from the largest reservation of the
// launch's blocks.
#pragma once

#include <type_traits>

#include "hm_aca_impl.cuh"

namespace hm {

namespace {

// Gaussian and Matern-3/2 kernels in float through exp2: the exponent's
// constant carries the factor log2(e) (rounded once, on the host), so an
// entry costs one multiply and one ex2 in place of the range reduction of
// expf; the rounding of the product D2 c is of the same order as the
// rounding of D2 c before expf.
// The Matern kernel of order 1 is a call (its series and quadrature would be
// inlined at every unrolled entry otherwise).
__device__ __noinline__ float matern_k1_call(float t) { return matern_k1(t); }
__device__ __noinline__ double matern_k1_call(double t) { return matern_k1(t); }

template <int KERN>
__device__ __forceinline__ float phi_team(float D2, float c, float c2)
{
    if (KERN == HM_GAUSSIAN) return exp2f(-(D2 * c2));
    if (KERN == HM_MATERN_K1) return matern_k1_call(D2 * c);
    const float s = sqrtf(D2);
    return fmaf(s, c, 1.0f) * exp2f(-(s * c2));
}

template <int KERN>
__device__ __forceinline__ double phi_team(double D2, double c, double)
{
    if (KERN == HM_MATERN_K1) return matern_k1_call(D2 * c);
    return phi<KERN>(D2, c);
}

template <class T>
struct TeamConst;
template <>
struct TeamConst<float> {
    static __host__ float c2(const KernelParams& kp)
    {
        // log2(e) folded into the exponent's constant
        return (float)((kp.kernel == HM_GAUSSIAN || kp.kernel == HM_MATERN32)
                           ? kp.c64 * 1.4426950408889634 : kp.c64);
    }
};
template <>
struct TeamConst<double> {
    static __host__ double c2(const KernelParams& kp) { return kp.c64; }
};

// Team barrier: the warp itself for W = 1, else a named barrier over the
// team's warps (ids 1.. per team; 0 is __syncthreads).
template <int W>
__device__ __forceinline__ void team_sync(int bar)
{
    if (W == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(32 * W) : "memory");
    }
}

// Values reduced over a team in one step: two compensated sums, a maximum
// of non-negative values, an argmax of |value| (ties to the lowest index)
// with its signed value, a minimum index, and a value held by one thread.
template <class T>
struct TRed {
    TSum<T> s0, s1;
    T x0;         // maximum, >= 0
    T av, aval;   // argmax: |value| (>= 0) and the signed value
    int ai;       // argmax index (INT_MAX: none)
    int mn;       // minimum index (INT_MAX: none)
    T pick;       // the value of the one thread that sets it, 0 elsewhere
    __device__ __forceinline__ void init()
    {
        s0.init();
        s1.init();
        x0 = av = aval = pick = T(0);
        ai = mn = 0x7fffffff;
    }
    __device__ __forceinline__ void take(T x, T v, int i)
    {
        if (x > av || (x == av && i < ai)) {
            av = x;
            aval = v;
            ai = i;
        }
    }
    __device__ __forceinline__ void join(const TRed& o)
    {
        s0.join(o.s0);
        s1.join(o.s1);
        x0 = max(x0, o.x0);
        take(o.av, o.aval, o.ai);
        mn = min(mn, o.mn);
        pick += o.pick;
    }
};

// Which fields a reduction carries.
enum { RD_SUMS = 1, RD_ARG = 2, RD_MN = 4, RD_PICK = 8 };

// Warp part of a reduction; every lane receives the warp's result. In float
// the maxima, the argmax and the minimum index are single warp-reduce
// instructions on the bit patterns (non-negative floats order like their
// bits); the owner of an entry index e is lane e mod 32. pick_lane is the
// lane that may hold pick.
template <int F>
__device__ __forceinline__ void warp_red(TRed<float>& q, int pick_lane)
{
    constexpr unsigned FULL = 0xffffffffu;
    if (F & RD_SUMS) {
        // a plain butterfly: 32 lane partials add with a relative error of
        // at most 5 roundings, far below what the stopping test resolves
        float a0 = q.s0.s + q.s0.c, a1 = q.s1.s + q.s1.c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(FULL, a0, o);
            a1 += __shfl_xor_sync(FULL, a1, o);
        }
        q.s0.set(a0);
        q.s1.set(a1);
    }
    q.x0 = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(q.x0)));
    if (F & RD_ARG) {
        const unsigned vb = __reduce_max_sync(FULL, __float_as_uint(q.av));
        const int w = __reduce_min_sync(FULL, __float_as_uint(q.av) == vb ? q.ai : 0x7fffffff);
        q.aval = __shfl_sync(FULL, q.aval, w & 31);
        q.av = __uint_as_float(vb);
        q.ai = w;
    }
    if (F & RD_MN) q.mn = __reduce_min_sync(FULL, q.mn);
    if (F & RD_PICK) q.pick = __shfl_sync(FULL, q.pick, pick_lane);
}

template <int F>
__device__ __forceinline__ void warp_red(TRed<double>& q, int pick_lane)
{
    constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (F & RD_SUMS) {
            q.s0.shfl_join(o);
            q.s1.shfl_join(o);
        }
        q.x0 = max(q.x0, __shfl_xor_sync(FULL, q.x0, o));
        if (F & RD_ARG) {
            const double oav = __shfl_xor_sync(FULL, q.av, o);
            const double oaval = __shfl_xor_sync(FULL, q.aval, o);
            const int oai = __shfl_xor_sync(FULL, q.ai, o);
            q.take(oav, oaval, oai);
        }
        if (F & RD_MN) q.mn = min(q.mn, __shfl_xor_sync(FULL, q.mn, o));
    }
    if (F & RD_PICK) q.pick = __shfl_sync(FULL, q.pick, pick_lane);
}

// Combination of up to 32 warp results held one per lane (lanes past the
// team's warps hold the identity): every lane receives the total. Used for
// teams of 8 or more warps in place of a join loop over the slots.
template <int F>
__device__ __forceinline__ void lane_join(TRed<float>& q)
{
    constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (F & RD_SUMS) {
            q.s0.shfl_join(o);
            q.s1.shfl_join(o);
        }
        if (F & RD_PICK) q.pick += __shfl_xor_sync(FULL, q.pick, o);
    }
    q.x0 = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(q.x0)));
    if (F & RD_ARG) {
        const unsigned vb = __reduce_max_sync(FULL, __float_as_uint(q.av));
        const bool cand = __float_as_uint(q.av) == vb;
        const int w = __reduce_min_sync(FULL, cand ? q.ai : 0x7fffffff);
        const unsigned who = __ballot_sync(FULL, cand && q.ai == w);
        q.aval = __shfl_sync(FULL, q.aval, who ? __ffs(who) - 1 : 0);
        q.av = __uint_as_float(vb);
        q.ai = w;
    }
    if (F & RD_MN) q.mn = __reduce_min_sync(FULL, q.mn);
}

template <int F>
__device__ __forceinline__ void lane_join(TRed<double>& q)
{
    constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (F & RD_SUMS) {
            q.s0.shfl_join(o);
            q.s1.shfl_join(o);
        }
        if (F & RD_PICK) q.pick += __shfl_xor_sync(FULL, q.pick, o);
        q.x0 = max(q.x0, __shfl_xor_sync(FULL, q.x0, o));
        if (F & RD_ARG) {
            const double oav = __shfl_xor_sync(FULL, q.av, o);
            const double oaval = __shfl_xor_sync(FULL, q.aval, o);
            const int oai = __shfl_xor_sync(FULL, q.ai, o);
            q.take(oav, oaval, oai);
        }
        if (F & RD_MN) q.mn = min(q.mn, __shfl_xor_sync(FULL, q.mn, o));
    }
}

// Per-team shared memory (dynamic, KT chosen at launch).
template <class T>
struct TeamSmem {
    T* Gu;      // packed Gram matrix of the u's, KT (KT + 1) / 2
    T* Gv;      // packed Gram matrix of the v's
    T* sgv;     // (v_l)_j of the current step, KT
    T* sgu;     // (u_l)_{i*} (or (u_l)_{iref}), KT
    T* dotw;    // per-warp partial dots, 2 x W x KT (column, row side)
    TRed<T>* slot;   // reduction slots, 2 x W
    StopState* st;   // the stopping test's state (thread 0 of the team)
    int* ctl;   // decisions of the step: resolved, stop_ok
};

__host__ __device__ constexpr size_t team_align(size_t b) { return (b + 15) & ~size_t(15); }

template <class T>
__host__ __device__ inline size_t team_smem_bytes(int W, int KT)
{
    const size_t ktp = (size_t)KT * (KT + 1) / 2;
    return team_align(2 * ktp * sizeof(T)) + team_align(2 * KT * sizeof(T)) +
           team_align((size_t)2 * W * KT * sizeof(T)) + team_align(2 * W * sizeof(TRed<T>)) +
           team_align(sizeof(StopState)) + 16;
}

template <class T>
__device__ __forceinline__ TeamSmem<T> team_carve(unsigned char* base, int W, int KT)
{
    TeamSmem<T> s;
    const size_t ktp = (size_t)KT * (KT + 1) / 2;
    unsigned char* p = base;
    s.Gu = reinterpret_cast<T*>(p);
    s.Gv = s.Gu + ktp;
    p += team_align(2 * ktp * sizeof(T));
    s.sgv = reinterpret_cast<T*>(p);
    s.sgu = s.sgv + KT;
    p += team_align(2 * KT * sizeof(T));
    s.dotw = reinterpret_cast<T*>(p);
    p += team_align((size_t)2 * W * KT * sizeof(T));
    s.slot = reinterpret_cast<TRed<T>*>(p);
    p += team_align(2 * W * sizeof(TRed<T>));
    s.st = reinterpret_cast<StopState*>(p);
    p += team_align(sizeof(StopState));
    s.ctl = reinterpret_cast<int*>(p);
    return s;
}

// Team-wide reduction: every thread of the team receives the result, joined
// over the warps in warp order. Slots are double buffered (ph): a later
// reduction writes the other buffer, and the one after that only once every
// thread has passed the barrier in between.
template <int F, class T, int W>
__device__ __forceinline__ TRed<T> team_reduce(TRed<T> q, const TeamSmem<T>& S, int& ph, int wt,
                                               int lane, int bar, int pick_lane = 0)
{
    warp_red<F>(q, pick_lane);
    if (W == 1) {
        __syncwarp();   // orders the lanes' shared-memory writes of the pass
        return q;
    }
    TRed<T>* sl = S.slot + ph * W;
    if (lane == 0) sl[wt] = q;
    team_sync<W>(bar);
    TRed<T> t;
    if (W >= 8) {
        if (lane < W) t = sl[lane];
        else t.init();
        lane_join<F>(t);
    } else {
        t = sl[0];
#pragma unroll
        for (int k = 1; k < W; ++k) t.join(sl[k]);
    }
    ph ^= 1;
    return t;
}

// Resident CTAs per SM asked of the register allocator: the small shapes
// are latency-bound and want many warps; the large ones keep 2 R residual
// entries and their loads in flight in registers.
template <class T, int W, int R>
__host__ __device__ constexpr int team_min_ctas()
{
    // 128-thread CTAs up to W = 4, one team of W warps above; float teams of
    // up to 4 warps with 8 entries per thread fit 96 registers (20 warps per
    // SM in place of 16)
    return W > 4 ? (W == 8 && R <= 16 ? 2 : 1)
                 : R <= 4 ? 6 : (R <= 8 && sizeof(T) == 4) ? 5 : R <= 16 ? 4 : 2;
}
// Threads of a CTA: 4 warps, or one team of W warps.
template <int W>
__host__ __device__ constexpr int team_cta_threads()
{
    return 32 * (W < 4 ? 4 : W);
}

// Residual pass of one side: entries uh[q] (index g + q G < len, zero
// elsewhere) minus sum_l s_l F_l (F_l the l-th factor column, length len,
// s_l held by lane l mod 32 of every warp in coef[l / 32]), in batches of LC ranks with the dots uh . F_l taken before
// each batch is subtracted (the partial residuals of the Gram correction);
// the warp's dot partials of rank l go to dotw[l]. Every load reads a valid
// entry (indices past len are clamped to len - 1) so that the loads of a
// batch issue together; the padding entries are reset to zero after each
// batch.
template <class T, int W, int R, bool DOTS>
__device__ __forceinline__ void team_resid(T (&uh)[R], const T* __restrict__ F, int len, int r,
                                           const T (&coef)[2], T* dotw, int g, int lane)
{
    constexpr int G = 32 * W;
    for (int l0 = 0; l0 < r; l0 += LC) {
        T sv[LC], p[LC];
        const T* Fb[LC];
        const T cw = l0 < 32 ? coef[0] : coef[1];   // lane l holds s_l, s_{l+32}
#pragma unroll
        for (int e = 0; e < LC; ++e) {
            sv[e] = __shfl_sync(0xffffffffu, cw, (l0 + e) & 31);
            p[e] = T(0);
            Fb[e] = F + (l0 + e < r ? (l0 + e) : l0) * len;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            // at most 8 entries' loads in flight per batch: a compiler fence
            // between groups of 8 keeps the loads of the next group from
            // being hoisted (they would need 4 registers per entry)
            if (q > 0 && q % 8 == 0) asm volatile("" ::: "memory");
            const bool ok = g + q * G < len;
            const int ix = ok ? g + q * G : len - 1;
            T u[LC];
#pragma unroll
            for (int e = 0; e < LC; ++e) u[e] = Fb[e][ix];
            if (DOTS) {
#pragma unroll
                for (int e = 0; e < LC; ++e) p[e] = fma(uh[q], u[e], p[e]);
            }
#pragma unroll
            for (int e = 0; e < LC; ++e) uh[q] = fma(-u[e], sv[e], uh[q]);
            uh[q] = ok ? uh[q] : T(0);
        }
        if (DOTS) {
            const T ps = warp_scatter(p);
            const int e = scatter_elem(lane);
            if (scatter_writer(lane) && l0 + e < r) dotw[l0 + e] = ps;
        }
    }
}

// Squared distance from p0 to the point in Morton row `row`, over the first
// D coordinate planes only (the planes above the sets' dimension hold zeros;
// their terms would add exact zeros, so the result is bit for bit that of
// dist2 over three planes).
template <int D>
__device__ __forceinline__ float dist2_planes(const Pt<float>& a, const DeviceCoords& X, int64_t row)
{
    const float* F = X.x32;
    const int64_t st = X.stride32;
    float t[3];
#pragma unroll
    for (int i = 0; i < D; ++i)
        t[i] = (a.h[i] - F[(2 * i) * st + row]) + (a.l[i] - F[(2 * i + 1) * st + row]);
    float r = t[0] * t[0];
#pragma unroll
    for (int i = 1; i < D; ++i) r = fmaf(t[i], t[i], r);
    return r;
}

template <int D>
__device__ __forceinline__ double dist2_planes(const Pt<double>& a, const DeviceCoords& X, int64_t row)
{
    double t[3];
#pragma unroll
    for (int i = 0; i < D; ++i) t[i] = a.x[i] - X.x64[i][row];
    double r = t[0] * t[0];
#pragma unroll
    for (int i = 1; i < D; ++i) r = fma(t[i], t[i], r);
    return r;
}

// The same pass in float on packed pairs of entries (q, q + 1): each
// residual entry takes the same fused multiply-adds in the same order
// (fma(u, -s, w) rounds like fma(-u, s, w)); the dots keep two partial sums,
// joined before the warp's reduce-scatter.
template <int W, int R, bool DOTS>
__device__ __forceinline__ void team_resid_f2(float (&uh)[R], const float* __restrict__ F, int len,
                                           int r, const float (&coef)[2], float* dotw, int g,
                                           int lane)
{
    constexpr int G = 32 * W;
    static_assert(R % 2 == 0, "entries in pairs");
    for (int l0 = 0; l0 < r; l0 += LC) {
        float2 ns[LC], p2[LC];
        const float* Fb[LC];
        const float cw = l0 < 32 ? coef[0] : coef[1];
#pragma unroll
        for (int e = 0; e < LC; ++e) {
            const float sv = __shfl_sync(0xffffffffu, cw, (l0 + e) & 31);
            ns[e] = make_float2(-sv, -sv);
            p2[e] = make_float2(0.f, 0.f);
            Fb[e] = F + (l0 + e < r ? (l0 + e) : l0) * len;
        }
#pragma unroll
        for (int q = 0; q < R; q += 2) {
            const bool ok0 = g + q * G < len, ok1 = g + (q + 1) * G < len;
            const int i0 = ok0 ? g + q * G : len - 1, i1 = ok1 ? g + (q + 1) * G : len - 1;
            float2 w = make_float2(uh[q], uh[q + 1]);
            float2 u[LC];
#pragma unroll
            for (int e = 0; e < LC; ++e) u[e] = make_float2(Fb[e][i0], Fb[e][i1]);
            if (DOTS) {
#pragma unroll
                for (int e = 0; e < LC; ++e) p2[e] = __ffma2_rn(w, u[e], p2[e]);
            }
#pragma unroll
            for (int e = 0; e < LC; ++e) w = __ffma2_rn(u[e], ns[e], w);
            uh[q] = ok0 ? w.x : 0.f;
            uh[q + 1] = ok1 ? w.y : 0.f;
        }
        if (DOTS) {
            float p[LC];
#pragma unroll
            for (int e = 0; e < LC; ++e) p[e] = p2[e].x + p2[e].y;
            const float ps = warp_scatter(p);
            const int e = scatter_elem(lane);
            if (scatter_writer(lane) && l0 + e < r) dotw[l0 + e] = ps;
        }
    }
}

template <class T, int W, int R, bool DOTS>
__device__ __forceinline__ void team_pass(T (&uh)[R], const T* __restrict__ F, int len, int r,
                                          const T (&coef)[2], T* dotw, int g, int lane)
{
    if constexpr (std::is_same<T, float>::value)
        team_resid_f2<W, R, DOTS>(uh, F, len, r, coef, dotw, g, lane);
    else
        team_resid<T, W, R, DOTS>(uh, F, len, r, coef, dotw, g, lane);
}

// Entries A(i, col0 + jj) of one row (or column: pass the other side's
// points) at the thread's indices g + q G < len, zero elsewhere; d2 selects
// the two-plane distance (sets of dimension 1 or 2).
template <class T, int KERN, int W, int R>
__device__ __forceinline__ void team_eval(T (&uh)[R], const DeviceCoords& X, const Pt<T>& p0,
                                          int64_t base, int len, int g, T c, T c2, bool d2)
{
    constexpr int G = 32 * W;
    if (d2) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const bool ok = g + q * G < len;
            const T v = phi_team<KERN>(dist2_planes<2>(p0, X, base + (ok ? g + q * G : 0)), c, c2);
            uh[q] = ok ? v : T(0);
        }
    } else {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const bool ok = g + q * G < len;
            const T v = phi_team<KERN>(dist2_planes<3>(p0, X, base + (ok ? g + q * G : 0)), c, c2);
            uh[q] = ok ? v : T(0);
        }
    }
}

template <class T, int KERN, int W, int R>
__global__ void __launch_bounds__(team_cta_threads<W>(), (team_min_ctas<T, W, R>()))
k_aca_team(KernelParams kp, DeviceCoords X, AcaArgs a, const uint32_t* __restrict__ order,
           int64_t nblocks, double thr, T c2, int KT)
{
    constexpr int G = 32 * W;
    constexpr int TPC = W < 4 ? 4 / W : 1;   // teams per CTA
    static_assert(R <= 32, "bit masks hold 32 entries per thread");
    extern __shared__ __align__(16) unsigned char team_dyn[];
    const int team = threadIdx.x / G;
    const int g = threadIdx.x - team * G;
    const int lane = threadIdx.x & 31, wt = g >> 5;
    const int bar = team + 1;
    const int64_t qb = (int64_t)blockIdx.x * TPC + team;
    if (qb >= nblocks) return;
    const TeamSmem<T> S = team_carve<T>(team_dyn + (size_t)team * team_smem_bytes<T>(W, KT), W, KT);

    const uint32_t b = order[qb];
    const Blk B = a.blk[b];
    const int m = B.m, n = B.n;
    const int kres = a.kres[b];
    const int kmax = min(kres, min(m, n));
    T* __restrict__ U = reinterpret_cast<T*>(a.Uptr[b]);
    T* __restrict__ V = reinterpret_cast<T*>(a.Vptr[b]);
    const T c = kconst<T>(kp);
    const T eps0 = (T)a.eps0;
    const bool d2 = kp.dmax <= 2;
    if (max(m, n) > R * G || kmax > KT) {   // the host routes no such block here
        if (g == 0) atomicOr(a.status, 2);
        return;
    }
    if (g == 0) {
        StopState st;
        const double rtol = a.eps > 0.0 ? a.eps : a.eps0;
        st.floor2 = a.bset ? (double)m * (double)n / (double)a.set_n[a.bset[b]] : 0.0;
        st.rtol2_m = rtol * rtol / (double)m;
        st.thr2 = thr * thr;
        st.fixed_rank = !(thr >= 0.0);
        *S.st = st;
    }
    int ph = 0;
    T uh[R], rr[R];
    unsigned used = 0u, seen = (g == 0) ? 1u : 0u;
    team_eval<T, KERN, W, R>(rr, X, load_pt<T>(X, B.row0), B.col0, n, g, c, c2, d2);   // reference row 0
    int r = 0, j = 0, rej = 0, run = 0, iref = 0;
    bool converged = false;
    const int limit = a.step_limit > 0 ? a.step_limit : kmax + n + 1;
    T du[2] = {T(0), T(0)};   // warp 0, lane l: u_r . u_l for l = lane, lane + 32
    T* dotw = S.dotw + wt * KT;
    for (int it = 0; r < kmax; ++it) {
        if (it > limit) {
            if (g == 0) atomicOr(a.status, 1);
            break;
        }
        if (j % G == g) used |= 1u << (j / G);
        // (v_l)_j of the earlier ranks: every warp loads them for itself
        // (lane l: ranks l and l + 32), warp 0 also keeps them for its Gram
        // correction
        T sreg[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int l = lane + 32 * s;
            sreg[s] = l < r ? V[l * n + j] : T(0);
            if (wt == 0 && l < KT) S.sgv[l] = sreg[s];
        }
        // ---- column pass: u^ = A(:, j) - sum_l u_l (v_l)_j, with w . u_l
        team_eval<T, KERN, W, R>(uh, X, load_pt<T>(X, B.col0 + j), B.row0, m, g, c, c2, d2);
        TRed<T> qc;
        qc.init();
#pragma unroll
        for (int q = 0; q < R; ++q) qc.x0 = max(qc.x0, fabs(uh[q]));
        team_pass<T, W, R, true>(uh, U, m, r, sreg, dotw, g, lane);
        {
            bool have_mn = false;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = g + q * G;
                if (i < m) {
                    qc.take(fabs(uh[q]), uh[q], i);
                    if (i == iref) qc.pick = uh[q];
                }
                if (!have_mn && i < n && !((used >> q) & 1u)) {
                    qc.mn = i;
                    have_mn = true;
                }
            }
        }
        const TRed<T> oc =
            team_reduce<RD_ARG | RD_MN | RD_PICK, T, W>(qc, S, ph, wt, lane, bar, iref & 31);
        if (!(oc.av > eps0 * oc.x0)) {
            // column already represented: take the lowest unused column, or
            // stop after rej_run rejections in a row
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
        // in float u_r = u^ / piv as products with 1 / piv, unless 1 / piv
        // would overflow (far blocks whose entries are near the underflow
        // limit); in double the quotients of Alg. 2 themselves, as the CPU
        // oracle forms them
        const bool small_piv = sizeof(T) == 8 || !(fabs(piv) >= T(1e-30));
        const T rpiv = small_piv ? T(0) : T(1) / piv;
        const int bi = oc.ai;
        const T uiref = small_piv ? oc.pick / piv : oc.pick * rpiv;
        if (bi % G == g) seen |= 1u << (bi / G);
        // warp 0: u_r . u_l = (w . u_l - sum_l' Gu(l, l') (v_l')_j) / piv;
        // then (u_l)_{i*} of the earlier ranks for the row pass
        if (wt == 0) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int l = lane + 32 * s;
                T x = T(0);
                if (l < r) {
#pragma unroll
                    for (int k = 0; k < W; ++k) x += S.dotw[k * KT + l];
                    for (int l2 = l - l % LC; l2 < r; ++l2)
                        x = fma(-S.Gu[l >= l2 ? pk(l, l2) : pk(l2, l)], S.sgv[l2], x);
                    x = small_piv ? x / piv : x * rpiv;
                }
                du[s] = x;
            }
        }
        // (u_l)_{i*} of the earlier ranks, per warp as above
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int l = lane + 32 * s;
            sreg[s] = l < r ? U[l * m + bi] : T(0);
            if (wt == 0 && l < KT) S.sgu[l] = sreg[s];
        }
        // u_r = u^ / piv
        TRed<T> qr;
        qr.init();
        {
            T* __restrict__ Ur = U + r * m + g;
            if (small_piv) {
#pragma unroll
                for (int q = 0; q < R; ++q) uh[q] = uh[q] / piv;
            } else {
#pragma unroll
                for (int q = 0; q < R; ++q) uh[q] = uh[q] * rpiv;
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (g + q * G < m) {
                    const T u = uh[q];
                    Ur[q * G] = u;
                    qr.s0.add(u * u);
                }
            }
        }
        // ---- row pass: v = A(i*, :) - sum_l (u_l)_{i*} v_l, with w . v_l
        // (its dot partials go to the second buffer: warp 0 may still read
        // the column pass's)
        team_eval<T, KERN, W, R>(uh, X, load_pt<T>(X, B.row0 + bi), B.col0, n, g, c, c2, d2);
        team_pass<T, W, R, true>(uh, V, n, r, sreg, dotw + W * KT, g, lane);
        {
            T* __restrict__ Vr = V + r * n + g;
            bool have_mn = false;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int jj = g + q * G;
                if (jj < n) {
                    const T v = uh[q];
                    Vr[q * G] = v;
                    qr.s1.add(v * v);
                    rr[q] = fma(-uiref, v, rr[q]);
                    const T x = fabs(rr[q]);
                    qr.x0 = max(qr.x0, x);
                    if (!((used >> q) & 1u)) qr.take(x, rr[q], jj);
                }
                if (!have_mn && jj < m && !((seen >> q) & 1u)) {
                    qr.mn = jj;
                    have_mn = true;
                }
            }
        }
        const TRed<T> orr = team_reduce<RD_SUMS | RD_ARG | RD_MN, T, W>(qr, S, ph, wt, lane, bar);
        // warp 0: v_l . v_r = w' . v_l - sum_l' Gv(l, l') (u_l')_{i*}; the
        // cross term of ||S_r||_F^2; Gram rows of rank r; the stopping test
        if (wt == 0) {
            T cr = T(0), dv[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int l = lane + 32 * s;
                T x = T(0);
                if (l < r) {
#pragma unroll
                    for (int k = 0; k < W; ++k) x += S.dotw[(W + k) * KT + l];
                    for (int l2 = l - l % LC; l2 < r; ++l2)
                        x = fma(-S.Gv[l >= l2 ? pk(l, l2) : pk(l2, l)], S.sgu[l2], x);
                }
                dv[s] = x;
                cr = fma(du[s], x, cr);
            }
            cr = warp_sum(cr);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int l = lane + 32 * s;
                if (l < r) {
                    S.Gu[pk(r, l)] = du[s];
                    S.Gv[pk(r, l)] = dv[s];
                }
            }
            if (lane == 0) {
                S.Gu[pk(r, r)] = orr.s0.rvalue();
                S.Gv[pk(r, r)] = orr.s1.rvalue();
                bool res, stp;
                stop_step(*S.st, orr.s0, orr.s1, cr, orr.x0, res, stp);
                S.ctl[0] = res;
                S.ctl[1] = stp;
            }
        }
        team_sync<W>(bar);
        ++r;
        bool resolved = S.ctl[0];
        const bool stop_ok = S.ctl[1];
        int nj = orr.ai;
        // a resolved reference row moves to the lowest row not seen yet
        if (resolved && orr.mn < m) {
            iref = orr.mn;
            if (iref % G == g) seen |= 1u << (iref / G);
            T sref[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int l = lane + 32 * s;
                sref[s] = l < r ? U[l * m + iref] : T(0);
            }
            team_eval<T, KERN, W, R>(uh, X, load_pt<T>(X, B.row0 + iref), B.col0, n, g, c, c2, d2);
            team_pass<T, W, R, false>(uh, V, n, r, sref, dotw, g, lane);
            TRed<T> qf;
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
            const TRed<T> of = team_reduce<RD_ARG, T, W>(qf, S, ph, wt, lane, bar);
            if (g == 0) S.ctl[0] = ref_resolved(*S.st, of.x0);
            team_sync<W>(bar);
            resolved = S.ctl[0];
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
        if (!converged && r >= kmax) f |= (kres < full) ? 1 : 2;   // re-run / rank cap
        a.flags[b] = f;
    }
}

template <class T, int KERN, int W, int R>
void launch_team(const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                 const uint32_t* order, int64_t n, double thr, int KT, cudaStream_t s)
{
    constexpr int NTH = team_cta_threads<W>();
    constexpr int TPC = W < 4 ? 4 / W : 1;
    auto kern = k_aca_team<T, KERN, W, R>;
    const size_t smem = TPC * team_smem_bytes<T>(W, KT);
    if (smem > 48 * 1024)
        HM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid = ceil_div(n, TPC);
    kern<<<(unsigned)grid, NTH, smem, s>>>(kp, X, a, order, n, thr, (T)TeamConst<T>::c2(kp), KT);
    note_launch();
}

// Team shapes (W warps, R entries per thread) per size class (class c:
// max(m, n) <= 64 << c). shape 1 is the default of the class: the fastest of
// the shapes measured on the 2-D Gaussian mixture at N = 2^20 (few entries
// per thread and more warps per block won from 512 rows on: the residuals
// and their loads in flight fit 128 registers, and the team's reductions
// amortise over more rows). The float Gaussian kernel also has the runner-up
// shapes compiled (shape 2), for measurements of the launch shape
// (hm_set_aca_shape). Returns false for a class or shape without a team
// kernel (the cluster kernels run).
template <class T, int KERN>
bool launch_team_class(const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                       const uint32_t* order, int64_t n, int cls, int shape, int KT,
                       cudaStream_t s)
{
    const double thr = (a.eps > 0.0) ? a.eps * (1.0 - a.aca_eta) / (1.0 + a.eps) : -1.0;
    constexpr bool alts = std::is_same<T, float>::value && KERN == HM_GAUSSIAN;
#define HM_TEAM(W_, R_) launch_team<T, KERN, W_, R_>(kp, X, a, order, n, thr, KT, s)
    const int key = cls * 4 + shape;
    switch (key) {
    case 0 * 4 + 1: HM_TEAM(1, 2); break;
    case 1 * 4 + 1: HM_TEAM(1, 4); break;
    case 2 * 4 + 1: HM_TEAM(1, 8); break;
    case 3 * 4 + 1: HM_TEAM(4, 4); break;
    case 4 * 4 + 1: HM_TEAM(4, 8); break;
    case 5 * 4 + 1: HM_TEAM(8, 8); break;
    case 6 * 4 + 1: HM_TEAM(16, 8); break;
    case 7 * 4 + 1: HM_TEAM(16, 16); break;
    case 8 * 4 + 1: HM_TEAM(32, 16); break;
    default:
        if constexpr (alts) {
            switch (key) {
            case 2 * 4 + 2: HM_TEAM(2, 4); break;
            case 3 * 4 + 2: HM_TEAM(2, 8); break;
            case 4 * 4 + 2: HM_TEAM(8, 4); break;
            case 5 * 4 + 2: HM_TEAM(16, 4); break;
            case 6 * 4 + 2: HM_TEAM(8, 16); break;
            case 7 * 4 + 2: HM_TEAM(32, 8); break;
            case 8 * 4 + 2: HM_TEAM(16, 32); break;
            default: return false;
            }
        } else {
            return false;
        }
    }
#undef HM_TEAM
    HM_LAUNCH("aca (team)");
    return true;
}

}  // namespace

}  // namespace hm
