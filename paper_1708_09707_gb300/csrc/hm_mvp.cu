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
// exactly once; x is gathered once (L2-resident reuse), y written once. The
// U slices and near-field slices a tile reads are contiguous (tile-major
// stores), and each gather entry carries its own descriptor, so the gather
// streams its data without dependent metadata loads.
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "hm_kernel_fn.cuh"
#include "hm_stream.cuh"

namespace hm {

namespace {

constexpr int NT = 256;
constexpr int VT_NT = 256;        // threads per CTA of the V^T x kernel
constexpr int TILE_NT = 256;      // threads per CTA of the gather kernel
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

// Reduce-scatter of four per-lane partial sums over the warp (a butterfly:
// the lane halves exchange two columns, then the quarters one, then the
// remaining lanes add one value): every lane returns the warp total of
// column (lane >> 3) & 3. Six additions per four columns instead of twenty
// for four separate warp sums, which matters where the additions share the
// FP64 pipe with the dot products.
template <class R>
__device__ __forceinline__ R warp_sum4(const R (&v)[4], int lane)
{
    const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
    R a0 = h16 ? v[2] : v[0], a1 = h16 ? v[3] : v[1];
    const R b0 = h16 ? v[0] : v[2], b1 = h16 ? v[1] : v[3];
    a0 += __shfl_xor_sync(0xffffffffu, b0, 16);
    a1 += __shfl_xor_sync(0xffffffffu, b1, 16);
    R c = h8 ? a1 : a0;
    const R e = h8 ? a0 : a1;
    c += __shfl_xor_sync(0xffffffffu, e, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// t partials: one warp per (block, 256-column chunk); lane j holds x of 8
// columns. Single precision reduces each factor column with its own warp
// sum; a chunk of at most 64 columns (the blocks of one leaf's width) takes
// two factor columns at once, one per half-warp. Double precision takes the columns four at a time, each lane summing
// its eight products per column, then one reduce-scatter (warp_sum4) per
// four columns: the additions share the FP64 pipe with the dot products, and
// this cuts them from five to 1.5 per column (measured at N = 2^20: 13.3 ms
// -> 10.0 ms; the same grouping made the single-precision kernel slower,
// 2.34 ms -> 3.33 ms, so it keeps the per-column sums).
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
    if (sizeof(R) == 4 && cn <= 64) {
        // chunks of at most 64 columns in float: half-warp h takes the ranks
        // l = h, h + 2, ..., lane j of it the columns j, j + 16, j + 32,
        // j + 48 (one running sum), then a butterfly over the half-warp
        const int h = lane >> 4, j = lane & 15;
        R xv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int jj = j + 16 * i;
            xv[i] = jj < cn ? xm[B.col0 + c0 + jj] : R(0);
        }
        const int64_t d = dst[w];
        R* out = d >= 0 ? tp + d : t + (-d - 1);
        for (int l0 = 0; l0 < k; l0 += 2) {
            const int l = l0 + h;
            R s = 0;
            if (l < k) {
                const R* Vl = V + (int64_t)l * n + c0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int jj = j + 16 * i;
                    if (jj < cn) s += Vl[jj] * xv[i];
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (j == 0 && l < k) out[l] = s;
        }
        return;
    }
    R xs[VCH / 32];
#pragma unroll
    for (int q = 0; q < VCH / 32; ++q) {
        const int jj = lane + 32 * q;
        xs[q] = (jj < cn) ? xm[B.col0 + c0 + jj] : R(0);
    }
    const int64_t d = dst[w];
    R* out = d >= 0 ? tp + d : t + (-d - 1);
    if constexpr (sizeof(R) == 8) {
        const int mine = (lane >> 3) & 3;
        for (int l0 = 0; l0 < k; l0 += 4) {
            R s[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                s[e] = R(0);
                if (l0 + e < k) {
                    const R* Vl = V + (int64_t)(l0 + e) * n + c0;
#pragma unroll
                    for (int q = 0; q < VCH / 32; ++q) {
                        const int jj = lane + 32 * q;
                        if (jj < cn) s[e] += Vl[jj] * xs[q];
                    }
                }
            }
            const R r = warp_sum4(s, lane);
            if ((lane & 7) == 0 && l0 + mine < k) out[l0 + mine] = r;
        }
    } else {
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


// Four consecutive rows of one slice column, from a 16-byte aligned address
// (streaming loads: every entry is read once per product).
__device__ __forceinline__ void ld4(const float* p, float (&o)[4])
{
    const float4 a = __ldcs(reinterpret_cast<const float4*>(p));
    o[0] = a.x;
    o[1] = a.y;
    o[2] = a.z;
    o[3] = a.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4])
{
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}


// Rows ir .. ir+3 of column c of a near-field stream starting at entry nb.
template <class R, int FMT>
__device__ __forceinline__ void near4(const void* store, int64_t nb, int64_t c, int ld, int ir,
                                      R (&o)[4])
{
    if (FMT == HM_NEAR_FP64) {
        double v[4];
        ld4(static_cast<const double*>(store) + nb + c * ld + ir, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = (R)v[i];
    } else if (FMT == HM_NEAR_FP32) {
        float v[4];
        ld4(static_cast<const float*>(store) + nb + c * ld + ir, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = (R)v[i];
    } else if (FMT == HM_NEAR_BF16X2) {
        const __nv_bfloat16* S = static_cast<const __nv_bfloat16*>(store) + 2 * nb + 2 * c * ld + ir;
        const uint2 h = __ldcs(reinterpret_cast<const uint2*>(S));
        const uint2 l = __ldcs(reinterpret_cast<const uint2*>(S + ld));
        const float2 h0 = bf2(h.x), h1 = bf2(h.y), l0 = bf2(l.x), l1 = bf2(l.y);
        o[0] = (R)(h0.x + l0.x);
        o[1] = (R)(h0.y + l0.y);
        o[2] = (R)(h1.x + l1.x);
        o[3] = (R)(h1.y + l1.y);
    } else {
        const __nv_bfloat16* S = static_cast<const __nv_bfloat16*>(store) + nb + c * ld + ir;
        const uint2 h = __ldcs(reinterpret_cast<const uint2*>(S));
        const float2 h0 = bf2(h.x), h1 = bf2(h.y);
        o[0] = (R)h0.x;
        o[1] = (R)h0.y;
        o[2] = (R)h1.x;
        o[3] = (R)h1.y;
    }
}

constexpr int T2_HW = TILE_NT / 16;   // half-warps per CTA

// Multiply-accumulate one column stream of a tile: half-warp hw takes
// columns hw, hw + 16, hw + 32, ..., TB at a time; lane hl < TB of the
// half-warp fetches the multiplier of the batch's column hl one batch ahead
// (its index and its value are two dependent loads), and passes it by a
// shuffle when the batch's data has arrived.
template <class R, int TB, class LD, class MUL>
__device__ __forceinline__ void tile_stream(int64_t cb, int64_t ncols, int hw, int hl, unsigned hmask,
                                            bool act, const LD& load_col, const MUL& mult,
                                            Acc<R> (&acc)[4])
{
    int64_t c0 = cb + hw;
    R mv = (hl < TB && c0 + 16 * hl < ncols) ? mult(c0 + 16 * hl) : R(0);
    for (; c0 < ncols; c0 += 16 * TB) {
        R a[TB][4];
#pragma unroll
        for (int e = 0; e < TB; ++e) {
            const int64_t c = c0 + 16 * e;
            if (act && c < ncols) load_col(c, a[e]);
            else a[e][0] = a[e][1] = a[e][2] = a[e][3] = R(0);
        }
        const int64_t cn = c0 + 16 * TB + 16 * hl;
        const R mnext = (hl < TB && cn < ncols) ? mult(cn) : R(0);
        if constexpr (sizeof(R) == 8) {
            // double: one running sum per row, column after column (the
            // FP64 pipe bounds this kernel, so no extra addition per group)
#pragma unroll
            for (int e = 0; e < TB; ++e) {
                const R m = __shfl_sync(hmask, mv, e, 16);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i].s = fma(a[e][i], m, acc[i].s);
            }
        } else {
            // plain sums over groups of four columns, each added compensated:
            // the grouping, hence the result, is the same for every TB
#pragma unroll
            for (int e0 = 0; e0 < TB; e0 += 4) {
                R sg[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
                for (int e = e0; e < e0 + 4; ++e) {
                    const R m = __shfl_sync(hmask, mv, e, 16);
#pragma unroll
                    for (int i = 0; i < 4; ++i) sg[i] = fma(a[e][i], m, sg[i]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i].add(sg[i]);
            }
        }
        mv = mnext;
    }
}

// One CTA per work item, a piece of one row tile's column stream: the tile's
// U slices followed by its near-field slices, slice_ld rows per column.
// Half-warp h takes the item's columns h, h + 16, h + 32, ... of each part,
// TB at a time, lane l of the half-warp rows 4l .. 4l+3 of the current
// 64-row window with one 16-byte load per column (two 8-byte loads for
// bfloat16 pairs). Every half-warp keeps compensated sums for its four rows,
// adding the plain sum of every four columns; the 16 partial sums of a row
// are added in half-warp order into the item's partial row sums. So the
// product is deterministic and the same for every TB (columns in flight per
// half-warp, a multiple of four) and MINB (CTAs per SM), the parameters the
// tuner picks.
template <class R, int FMT, int TB, int MINB>
__global__ void __launch_bounds__(TILE_NT, MINB)
k_tile(MvpPlan P, const R* __restrict__ xm, const R* __restrict__ t, double* __restrict__ part)
{
    __shared__ double ps[T2_HW][TROWS];
    const int64_t item = blockIdx.x;
    const int3 it = P.items[item];
    const int64_t tile = it.x;
    const int hw = threadIdx.x >> 4, hl = threadIdx.x & 15;
    const unsigned hmask = 0xffffu << (threadIdx.x & 16);
    const int mt = P.tile_m[tile];
    const int ld = slice_ld(mt);
    const int64_t uc0 = P.ucol_ptr[tile], nu = P.ucol_ptr[tile + 1] - uc0, ub = P.ubase[tile];
    const int64_t nc0 = P.ncol_ptr[tile], nb = P.nbase[tile];
    // the item's part of each stream
    const int64_t ucb = it.y < nu ? it.y : nu, uce = it.z < nu ? it.z : nu;
    const int64_t ncb = it.y > nu ? it.y - nu : 0, nce = it.z > nu ? it.z - nu : 0;
    const R* __restrict__ US = static_cast<const R*>(P.ustore);
    const int32_t* __restrict__ ucol_t = P.ucol_t;
    const int32_t* __restrict__ ncol_x = P.ncol_x;
    const void* __restrict__ near = P.near;
    double* __restrict__ out = part + item * P.max_ld;
    for (int rp = 0; rp < ld; rp += TROWS) {
        const int ir = rp + 4 * hl;
        const bool act = ir < ld;
        Acc<R> acc[4];
        tile_stream<R, TB>(
            ucb, uce, hw, hl, hmask, act,
            [&](int64_t c, R(&o)[4]) { ld4(US + ub + c * ld + ir, o); },
            [&](int64_t c) { return t[ucol_t[uc0 + c]]; }, acc);
        tile_stream<R, TB>(
            ncb, nce, hw, hl, hmask, act,
            [&](int64_t c, R(&o)[4]) { near4<R, FMT>(near, nb, c, ld, ir, o); },
            [&](int64_t c) { return xm[ncol_x[nc0 + c]]; }, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i) ps[hw][4 * hl + i] = act ? acc[i].value() : 0.0;
        __syncthreads();
        const int rows = min(TROWS, mt - rp);
        if ((int)threadIdx.x < rows) {
            double sum = 0.0;
#pragma unroll
            for (int q = 0; q < T2_HW; ++q) sum += ps[q][threadIdx.x];
            out[rp + threadIdx.x] = sum;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ bulk-copy gather
// The same work item as k_tile, with its column streams moved into shared
// memory by the bulk-copy (TMA) engine: one producer thread issues one
// cp.async.bulk per chunk of TCOL columns (a contiguous run of TCOL columns
// of slice_ld entries) into a ring of TS stages; 8 consumer warps fetch each
// chunk's multipliers one chunk ahead, wait on the stage's mbarrier,
// multiply and release the stage. Half-warp h takes the chunk's columns h, h + 16, ...
// (the columns h, h + 16, h + 32, ... of the stream, as in k_tile), and the
// plain sums run over the same groups of four columns, so the result is
// bit-for-bit that of k_tile. Only for slices of at most 64 rows (one row
// window).
constexpr int T3_CONS = 8;             // consumer warps
constexpr int T3_NT = (T3_CONS + 1) * 32;

template <class R, int FMT>
__host__ __device__ constexpr int col_bytes64()   // bytes of one 64-row column
{
    return FMT == HM_NEAR_FP64 ? (sizeof(R) > 8 ? 0 : 512)
           : (sizeof(R) == 8 ? 512 : 256);
}

// Reduce-scatter of four per-lane values over a half-warp: every lane
// returns the half-warp total of value (hl >> 2) & 3 (hl the lane's index in
// its half-warp). Both half-warps run it together.
template <class R>
__device__ __forceinline__ R halfwarp_sum4(const R (&v)[4], int hl)
{
    const bool b3 = (hl & 8) != 0, b2 = (hl & 4) != 0;
    R a0 = b3 ? v[2] : v[0], a1 = b3 ? v[3] : v[1];
    const R s0 = b3 ? v[0] : v[2], s1 = b3 ? v[1] : v[3];
    a0 += __shfl_xor_sync(0xffffffffu, s0, 8);
    a1 += __shfl_xor_sync(0xffffffffu, s1, 8);
    R c = b2 ? a1 : a0;
    const R e = b2 ? a0 : a1;
    c += __shfl_xor_sync(0xffffffffu, e, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// ZT (symmetric near field): a near column c of the tile's stream also
// gives (A^T x|tile)_c = sum over the tile's rows of A(row, c) x(row), the
// row-c entry of the mirror leaf's product, written to P.zbuf at the
// column's index in the near stream; with P.zubuf (pass A of the symmetric
// low-rank part) every U column likewise gives (U_b^T x|tile)_l, written at
// its index in the U stream.
template <class R, int FMT, int TCOL, int TS, bool ZT = false>
__global__ void __launch_bounds__(T3_NT, (ZT || TCOL == 128) ? 3 : 2)
k_tile_tma(MvpPlan P, const R* __restrict__ xm, const R* __restrict__ t, double* __restrict__ part)
{
    extern __shared__ __align__(128) unsigned char tsm[];
    constexpr int STAGE = TCOL * col_bytes64<R, FMT>();
    __shared__ uint64_t full[TS], empty[TS];
    static_assert(TCOL == 32 || TCOL == 64 || TCOL == 128, "32, 64 or 128 columns per stage");
    __shared__ double ps[T2_HW][TROWS];
    __shared__ int failed;
    const int64_t item = blockIdx.x;
    const int3 it = P.items[item];
    const int64_t tile = it.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = P.tile_m[tile];
    const int ld = slice_ld(mt);
    int64_t uc0 = P.ucol_ptr[tile], nu = P.ucol_ptr[tile + 1] - uc0, ub = P.ubase[tile];
    if (P.umid) {
        // symmetric low-rank part: pass A streams the canonical slices (and
        // the near field), pass B the mirror slices
        const int64_t um = P.umid[tile];
        if (P.uview == 2) {
            ub += (um - uc0) * ld;
            nu -= um - uc0;
            uc0 = um;
        } else {
            nu = um - uc0;
        }
    }
    const int64_t nc0 = P.ncol_ptr[tile], nb = P.nbase[tile];
    const int64_t ucb = it.y < nu ? it.y : nu, uce = it.z < nu ? it.z : nu;
    const int64_t ncb = it.y > nu ? it.y - nu : 0, nce = it.z > nu ? it.z - nu : 0;
    const int nuch = (int)ceil_div(uce - ucb, TCOL), nnch = (int)ceil_div(nce - ncb, TCOL);
    const int nch = nuch + nnch;
    // bytes of one column of the U stream and of the near-field stream
    const int ucolb = ld * (int)sizeof(R);
    const int ncolb = FMT == HM_NEAR_FP64 ? ld * 8 : FMT == HM_NEAR_FP32 ? ld * 4
                    : FMT == HM_NEAR_BF16X2 ? ld * 4 : ld * 2;
    if (threadIdx.x == 0) {
        for (int k = 0; k < TS; ++k) {
            mbar_init(&full[k], 1);         // the producer's arrival with the byte count
            mbar_init(&empty[k], T3_CONS);  // one arrival per consumer warp
        }
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // chunk k: stream part, first column and column count
    auto chunk = [&](int k, bool& isu, int64_t& c0, int& cnt) {
        isu = k < nuch;
        c0 = isu ? ucb + (int64_t)k * TCOL : ncb + (int64_t)(k - nuch) * TCOL;
        const int64_t cend = isu ? uce : nce;
        cnt = (int)(cend - c0 < TCOL ? cend - c0 : TCOL);
    };
    if (w == T3_CONS) {
        // ---------------- producer: one thread issues the copies
        if (lane == 0) {
            int k = 0;
            for (; k < nch; ++k) {
                const int slot = k % TS;
                if (k >= TS && !mbar_wait(&empty[slot], ((k / TS) - 1) & 1, P.wait_ns)) {
                    atomicOr(P.status, 4);
                    break;
                }
                bool isu;
                int64_t c0;
                int cnt;
                if (k == P.withhold) continue;   // test hook: this chunk never arrives
                chunk(k, isu, c0, cnt);
                const uint32_t bytes = (uint32_t)(cnt * (isu ? ucolb : ncolb));
                const char* src = isu
                    ? reinterpret_cast<const char*>(static_cast<const R*>(P.ustore) + ub + c0 * ld)
                    : static_cast<const char*>(P.near) + (int64_t)ncolb * c0 +
                          (FMT == HM_NEAR_BF16X2 ? 4 * nb : FMT == HM_NEAR_BF16 ? 2 * nb
                           : FMT == HM_NEAR_FP32 ? 4 * nb : 8 * nb);
                mbar_arrive_tx(&full[slot], bytes);
                bulk_copy(tsm + slot * STAGE, src, bytes, &full[slot]);
            }
            // every copy issued lands before the CTA exits: only the last TS
            // chunks issued can still be in flight, and a wait on a phase
            // that has completed returns at once
            for (int q = (k > TS ? k - TS : 0); q < k; ++q)
                if (q != P.withhold &&
                    !mbar_wait(&full[q % TS], (q / TS) & 1, P.wait_ns > MBAR_DRAIN_NS ? P.wait_ns : MBAR_DRAIN_NS))
                    atomicOr(P.status, 4);
        }
    } else {
        // ---------------- consumers: half-warp hw = 2w + (lane >> 4)
        const int hw = threadIdx.x >> 4, hl = threadIdx.x & 15;
        const unsigned hmask = 0xffffu << (threadIdx.x & 16);
        const int ir = 4 * hl;
        const bool act = ir < ld;
        constexpr int E = TCOL / 16;   // columns per half-warp and chunk
        // lane hl < E of the half-warp fetches the multiplier of the chunk's
        // column hw + 16 hl, one chunk ahead
        auto fetch = [&](int k) -> R {
            if (k >= nch || hl >= E) return R(0);
            bool isu;
            int64_t c0;
            int cnt;
            chunk(k, isu, c0, cnt);
            const int col = hw + 16 * hl;
            if (col >= cnt) return R(0);
            return isu ? t[P.ucol_t[uc0 + c0 + col]] : xm[P.ncol_x[nc0 + c0 + col]];
        };
        Acc<R> acc[4];
        R sg[4] = {R(0), R(0), R(0), R(0)};
        int ing = 0;   // columns of the current group of four
        R xr[4] = {R(0), R(0), R(0), R(0)};   // x of this lane's rows (ZT)
        if constexpr (ZT) {
            static_assert(TCOL / 16 == 4 || TCOL / 16 == 8, "four or eight columns per half-warp and chunk");
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (ir + i < mt) xr[i] = xm[P.tile_row0[tile] + ir + i];
        }
        R mv = fetch(0);
        for (int k = 0; k < nch; ++k) {
            const int slot = k % TS;
            const R mnext = fetch(k + 1);
            // the whole warp gives up together, so the shuffles below never
            // name a lane that has left
            if (!__all_sync(0xffffffffu, mbar_wait(&full[slot], (k / TS) & 1, P.wait_ns))) {
                if (lane == 0) atomicOr(P.status, 4);
                failed = 1;
                break;
            }
            bool isu;
            int64_t c0;
            int cnt;
            chunk(k, isu, c0, cnt);
            const unsigned char* st = tsm + slot * STAGE;
            R za[E];
#pragma unroll
            for (int e = 0; e < E; ++e) za[e] = R(0);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int col = hw + 16 * e;
                R a[4] = {R(0), R(0), R(0), R(0)};
                if (act && col < cnt) {
                    if (isu) {
                        const R* q = reinterpret_cast<const R*>(st + col * ucolb) + ir;
#pragma unroll
                        for (int i = 0; i < 4; ++i) a[i] = q[i];
                    } else if (FMT == HM_NEAR_BF16X2) {
                        const __nv_bfloat16* q = reinterpret_cast<const __nv_bfloat16*>(st + col * ncolb) + ir;
                        const uint2 h = *reinterpret_cast<const uint2*>(q);
                        const uint2 l = *reinterpret_cast<const uint2*>(q + ld);
                        const float2 h0 = bf2(h.x), h1 = bf2(h.y), l0 = bf2(l.x), l1 = bf2(l.y);
                        if constexpr (sizeof(R) == 4) {
                            // packed pairs: every entry rounds as hi + lo alone
                            const float2 s01 = __fadd2_rn(h0, l0), s23 = __fadd2_rn(h1, l1);
                            a[0] = s01.x;
                            a[1] = s01.y;
                            a[2] = s23.x;
                            a[3] = s23.y;
                        } else {
                            a[0] = (R)(h0.x + l0.x);
                            a[1] = (R)(h0.y + l0.y);
                            a[2] = (R)(h1.x + l1.x);
                            a[3] = (R)(h1.y + l1.y);
                        }
                    } else if (FMT == HM_NEAR_BF16) {
                        const __nv_bfloat16* q = reinterpret_cast<const __nv_bfloat16*>(st + col * ncolb) + ir;
                        const uint2 h = *reinterpret_cast<const uint2*>(q);
                        const float2 h0 = bf2(h.x), h1 = bf2(h.y);
                        a[0] = (R)h0.x;
                        a[1] = (R)h0.y;
                        a[2] = (R)h1.x;
                        a[3] = (R)h1.y;
                    } else if (FMT == HM_NEAR_FP32) {
                        const float* q = reinterpret_cast<const float*>(st + col * ncolb) + ir;
#pragma unroll
                        for (int i = 0; i < 4; ++i) a[i] = (R)q[i];
                    } else {
                        const double* q = reinterpret_cast<const double*>(st + col * ncolb) + ir;
#pragma unroll
                        for (int i = 0; i < 4; ++i) a[i] = (R)q[i];
                    }
                }
                const R m = __shfl_sync(hmask, mv, e, 16);
                if constexpr (sizeof(R) == 8) {
                    // double: one running sum per row, as in k_tile
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[i].s = fma(a[i], m, acc[i].s);
                } else {
                    // packed pairs of rows: every row takes the multiply-add
                    // it takes alone (the sums of k_tile, bit for bit)
                    const float2 mm = make_float2(m, m);
                    const float2 s01 = __ffma2_rn(make_float2(a[0], a[1]), mm, make_float2(sg[0], sg[1]));
                    const float2 s23 = __ffma2_rn(make_float2(a[2], a[3]), mm, make_float2(sg[2], sg[3]));
                    sg[0] = s01.x;
                    sg[1] = s01.y;
                    sg[2] = s23.x;
                    sg[3] = s23.y;
                }
                if constexpr (ZT) {
                    if (!isu || P.zubuf) {
                        if constexpr (sizeof(R) == 4) {
                            // rows (0, 2) and (1, 3) in two packed running
                            // sums, joined at the end
                            float2 zp = __fmul2_rn(make_float2(a[0], a[1]), make_float2(xr[0], xr[1]));
                            zp = __ffma2_rn(make_float2(a[2], a[3]), make_float2(xr[2], xr[3]), zp);
                            za[e] = zp.x + zp.y;
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i) za[e] = fma(a[i], xr[i], za[e]);
                        }
                    }
                }
                // groups of four columns of this half-warp's sequence, as in
                // k_tile; a stream part starts a new group
                const bool last = (k == nuch - 1 || k == nch - 1) && e == E - 1;
                if (sizeof(R) != 8 && (++ing == 4 || last)) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        acc[i].add(sg[i]);
                        sg[i] = R(0);
                    }
                    ing = 0;
                }
            }
            if constexpr (ZT) {
                if (!isu || P.zubuf) {
                    // one transposed product per column of the chunk (near
                    // columns: the mirror leaf's rows; U columns of pass A:
                    // the mirror block's t)
#pragma unroll
                    for (int g4 = 0; g4 < E / 4; ++g4) {
                        const R zq[4] = {za[4 * g4], za[4 * g4 + 1], za[4 * g4 + 2], za[4 * g4 + 3]};
                        const R z = halfwarp_sum4(zq, hl);
                        const int col = hw + 16 * (4 * g4 + ((hl >> 2) & 3));
                        if ((hl & 3) == 0 && col < cnt) {
                            if (isu) P.zubuf[uc0 + c0 + col] = (float)z;
                            else P.zbuf[nc0 + c0 + col] = (float)z;
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            mv = mnext;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) ps[hw][4 * hl + i] = act ? acc[i].value() : 0.0;
    }
    __syncthreads();
    if ((int)threadIdx.x < mt && !failed) {
        double sum = 0.0;
#pragma unroll
        for (int q = 0; q < T2_HW; ++q) sum += ps[q][threadIdx.x];
        part[item * P.max_ld + threadIdx.x] = sum;
    }
}

// y for every row of every tile: the tile's item sums in item order, plus
// sigma^2 x, written in the caller's order (one warp per tile).
__global__ void k_tile_finish(MvpPlan P, const double* __restrict__ part, const double* __restrict__ x,
                              double* __restrict__ y, int accumulate)
{
    const int64_t tile = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= P.n_tiles) return;
    const int64_t r0 = P.tile_row0[tile];
    const int mt = P.tile_m[tile];
    const int64_t i0 = P.item_ptr[tile], i1 = P.item_ptr[tile + 1];
    for (int i = lane; i < mt; i += 32) {
        double sum = 0.0;
        for (int64_t q = i0; q < i1; ++q) sum += part[q * P.max_ld + i];
        const int64_t row = r0 + i;
        const int64_t dst = P.perm[row];
        const double sg = P.sig_row ? P.sig_row[row] : P.sigma2;
        const double v = sum + sg * x[dst];
        y[dst] = accumulate ? y[dst] + v : v;
    }
}

// Symmetric low-rank part: t of every mirror block (sigma, tau) is U_b^T x|tau
// of its canonical partner b, the sum over b's slices (tile order) of the
// transposed products pass A wrote per U column; bmcol[e] is the first U
// column of b's block-major entry e. Blocks of at most 8 slices (most): one
// thread per block, column by column, the slices in order.
__global__ void k_tmirror_small(const int32_t* __restrict__ rank,
                                const int32_t* __restrict__ mirror_of,
                                const int64_t* __restrict__ boff, const int64_t* __restrict__ bmcol,
                                int64_t nlr, int64_t nb, const int64_t* __restrict__ toff,
                                const float* __restrict__ zu, float* __restrict__ t)
{
    const int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= nb) return;
    const int32_t m = mirror_of[b];
    if (m < 0) return;
    const int64_t e0 = boff[b], e1 = b + 1 < nb ? boff[b + 1] : nlr;
    if (e1 - e0 > 8) return;
    const int k = rank[b];
    for (int l = 0; l < k; ++l) {
        float sum = 0.f;
        for (int64_t e = e0; e < e1; ++e) sum += zu[bmcol[e] + l];
        t[toff[m] + l] = sum;
    }
}

// The canonical blocks of more than 8 slices (big[]): one warp per block;
// lane j sums the slices j, j + 32, ... of column l, then a warp sum.
__global__ void k_tmirror_big(const int32_t* __restrict__ big, int64_t nbig,
                              const int32_t* __restrict__ rank,
                              const int32_t* __restrict__ mirror_of,
                              const int64_t* __restrict__ boff, const int64_t* __restrict__ bmcol,
                              int64_t nlr, int64_t nb, const int64_t* __restrict__ toff,
                              const float* __restrict__ zu, float* __restrict__ t)
{
    const int64_t w = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nbig) return;
    const int b = big[w];
    const int32_t m = mirror_of[b];
    const int k = rank[b];
    const int64_t e0 = boff[b], e1 = b + 1 < nb ? boff[b + 1] : nlr;
    for (int l = 0; l < k; ++l) {
        float sum = 0.f;
        for (int64_t e = e0 + lane; e < e1; e += 32) sum += zu[bmcol[e] + l];
        sum = warp_sum(sum);
        if (lane == 0) t[toff[m] + l] = sum;
    }
}

// Canonical blocks with a mirror and more than 8 slices.
__global__ void k_big_flag(const int32_t* __restrict__ mirror_of, const int64_t* __restrict__ boff,
                           int64_t nlr, int64_t nb, int64_t* __restrict__ f)
{
    const int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= nb) return;
    const int64_t e1 = b + 1 < nb ? boff[b + 1] : nlr;
    f[b] = (mirror_of[b] >= 0 && e1 - boff[b] > 8) ? 1 : 0;
}

__global__ void k_big_ids(const int64_t* __restrict__ f, const int64_t* __restrict__ off,
                          int64_t nb, int32_t* __restrict__ ids)
{
    const int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b < nb && f[b]) ids[off[b]] = (int32_t)b;
}

// First U column of every block-major low-rank entry (through the CSR
// position of the entry).
__global__ void k_bm_ecol(const int64_t* __restrict__ pos, const int64_t* __restrict__ ecol,
                          int64_t n, int64_t* __restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e < n) out[e] = ecol[pos[e]];
}

// The finish of a symmetric near field (tiles of at most 64 rows): one CTA
// per tile, four groups of 64 threads (thread = row). Group g sums the
// mirror leaves' transposed products of records g, g + 4, ... in record
// order; row i then takes its item sums in item order and the four group
// sums in group order, plus sigma^2 x.
__global__ void __launch_bounds__(256)
k_tile_finish_sym(MvpPlan P, const double* __restrict__ part, const double* __restrict__ x,
                  double* __restrict__ y, int accumulate)
{
    __shared__ double zs[4][64];
    const int64_t tile = blockIdx.x;
    const int i = threadIdx.x & 63, g = threadIdx.x >> 6;
    const int mt = P.tile_m[tile];
    const int64_t z0 = P.zptr[tile], z1 = P.zptr[tile + 1];
    double s = 0.0;
    for (int64_t r = z0 + g; r < z1; r += 4)
        if (i < P.zlen[r]) s += (double)P.zbuf[P.zbase[r] + i];
    zs[g][i] = s;
    __syncthreads();
    if (g != 0 || i >= mt) return;
    const int64_t i0 = P.item_ptr[tile], i1 = P.item_ptr[tile + 1];
    double sum = 0.0;
    for (int64_t q = i0; q < i1; ++q) sum += part[q * P.max_ld + i];
    if (P.item_ptr_b) {
        // pass B's items (mirror slices), stored after pass A's
        const int64_t j0 = P.item_ptr_b[tile], j1 = P.item_ptr_b[tile + 1];
        for (int64_t q = j0; q < j1; ++q) sum += part[(P.n_items + q) * P.max_ld + i];
    }
    sum += zs[0][i];
    sum += zs[1][i];
    sum += zs[2][i];
    sum += zs[3][i];
    const int64_t row = P.tile_row0[tile] + i;
    const int64_t dst = P.perm[row];
    const double sg = P.sig_row ? P.sig_row[row] : P.sigma2;
    const double v = sum + sg * x[dst];
    y[dst] = accumulate ? y[dst] + v : v;
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
                               int32_t* __restrict__ tcount, const int32_t* __restrict__ cls)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= nb) return;
    const Blk B = blk[b];
    for (int64_t q = 0; q < cnt[b]; ++q) {
        int64_t e = off[b] + q, tl = first[b] + q;
        key[e] = cls ? 2 * (uint64_t)tl + (uint64_t)cls[b] : (uint64_t)tl;
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

__global__ void k_inverse_perm(const uint32_t* __restrict__ val, int64_t n, int64_t* __restrict__ pos)
{
    int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i < n) pos[val[i]] = i;
}

// Build one CSR over tiles for a list of blocks. Within a tile the entries
// keep block order; with cls (0 or 1 per block) the class-0 entries of a
// tile come first. boff/pos (optional): the first block-major entry of every
// block (its entries over its tiles are boff[b] .. boff[b] + count - 1, in
// tile order) and the CSR position of every block-major entry.
void build_csr(const Blk* blk, int64_t nb, const int64_t* tr0, int64_t nt,
               DevBuf<int64_t>& ptr, DevBuf<int2>& ent, cudaStream_t s,
               const int32_t* cls = nullptr, DevBuf<int64_t>* boff = nullptr,
               DevBuf<int64_t>* pos = nullptr)
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
                                               val.p, tmp.p, tcount.p, cls); note_launch();
    HM_LAUNCH("emit entries");
    radix_sort_u64_u32(key.p, val.p, E, bits_for(nt + 1) + (cls ? 1 : 0), s);
    ent.alloc(E, s);
    k_gather_ent<<<grid_for(E), NT, 0, s>>>(tmp.p, val.p, E, ent.p); note_launch();
    if (pos) {
        pos->alloc(E, s);
        k_inverse_perm<<<grid_for(E), NT, 0, s>>>(val.p, E, pos->p); note_launch();
    }
    if (boff) *boff = std::move(off);
    DevBuf<int64_t> c64(nt + 1, s);
    k_i32_to_i64<<<grid_for(nt + 1), NT, 0, s>>>(tcount.p, nt + 1, c64.p); note_launch();
    scan_exclusive_i64(c64.p, ptr.p, nt + 1, nullptr, s);
    HM_LAUNCH("csr");
}

// tile index of every CSR entry
__global__ void k_entry_tiles(const int64_t* __restrict__ ptr, int64_t nt, int32_t* __restrict__ et)
{
    const int64_t tl = blockIdx.x;
    if (tl >= nt) return;
    for (int64_t e = ptr[tl] + threadIdx.x; e < ptr[tl + 1]; e += blockDim.x) et[e] = (int32_t)tl;
}

__global__ void k_lr_sizes(const int2* __restrict__ ent, const int32_t* __restrict__ et,
                           int64_t ne, const int32_t* __restrict__ rank,
                           const int32_t* __restrict__ tile_m, int64_t* __restrict__ sz)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e < ne) sz[e] = (int64_t)rank[ent[e].x] * slice_ld(tile_m[et[e]]);
}

__global__ void k_lr_desc(const int2* __restrict__ ent, int64_t ne,
                          const int32_t* __restrict__ rank, const int64_t* __restrict__ off,
                          const int64_t* __restrict__ toff, LrDesc* __restrict__ d)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    const int b = ent[e].x;
    LrDesc q;
    q.uoff = off[e];
    q.toff = toff[b];
    q.k = rank[b];
    q.pad = 0;
    d[e] = q;
}

__global__ void k_dn_sizes(const int2* __restrict__ ent, const int32_t* __restrict__ et,
                           int64_t ne, const Blk* __restrict__ dblk,
                           const int32_t* __restrict__ tile_m, int64_t* __restrict__ sz)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e < ne) sz[e] = (int64_t)dblk[ent[e].x].n * slice_ld(tile_m[et[e]]);
}

__global__ void k_dn_desc(const int2* __restrict__ ent, int64_t ne, const Blk* __restrict__ dblk,
                          const int64_t* __restrict__ off, DnDesc* __restrict__ d)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    const Blk B = dblk[ent[e].x];
    DnDesc q;
    q.noff = off[e];
    q.col0 = B.col0;
    q.n = B.n;
    q.pad = 0;
    d[e] = q;
}

// One warp per low-rank entry: copy U_b(rowoff + 0..rows, 0..k) (leading
// dimension m_b) into the entry's slice (leading dimension rows).
template <class R>
__global__ void k_relayout_u(const int2* __restrict__ ent, const int32_t* __restrict__ et,
                             const LrDesc* __restrict__ desc, int64_t ne,
                             const Blk* __restrict__ ablk, const uint64_t* __restrict__ Uptr,
                             const int32_t* __restrict__ tile_m, R* __restrict__ dst)
{
    const int64_t w = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= ne) return;
    const int2 en = ent[w];
    const int rows = tile_m[et[w]];
    const int ld = slice_ld(rows);
    const int m = ablk[en.x].m;
    const LrDesc d = desc[w];
    const R* src = reinterpret_cast<const R*>(Uptr[en.x]) + en.y;
    R* out = dst + d.uoff;
    // 64 rows x 4 columns per round: eight loads in flight per lane
    for (int i0 = 0; i0 < ld; i0 += 64)
        for (int l0 = 0; l0 < d.k; l0 += 4) {
            R v[4][2];
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = i0 + lane + 32 * h, l = l0 + e;
                    v[e][h] = (l < d.k && i < rows) ? src[(int64_t)l * m + i] : R(0);
                }
#pragma unroll
            for (int e = 0; e < 4; ++e)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = i0 + lane + 32 * h, l = l0 + e;
                    if (l < d.k && i < ld) out[(int64_t)l * ld + i] = v[e][h];
                }
        }
}

__global__ void k_vitems_count(const Blk* __restrict__ blk, const int32_t* __restrict__ rank,
                               int64_t nb, int64_t* __restrict__ cnt,
                               int64_t* __restrict__ multi_t, int32_t* __restrict__ ismulti,
                               int64_t* __restrict__ rk, const int32_t* __restrict__ cls)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= nb) return;
    int k = rank[b];
    // (the symmetric low-rank part forms a mirror block's t in pass A)
    int64_t c = (k > 0 && !(cls && cls[b])) ? ceil_div(blk[b].n, VCH) : 0;
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

// Columns of every gather entry: the rank of its block (low-rank list) or
// the block's column count (dense list).
__global__ void k_lr_ncols(const int2* __restrict__ ent, int64_t ne, const int32_t* __restrict__ rank,
                           int64_t* __restrict__ cnt)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e < ne) cnt[e] = rank[ent[e].x];
}

__global__ void k_dn_ncols(const int2* __restrict__ ent, int64_t ne, const Blk* __restrict__ dblk,
                           int64_t* __restrict__ cnt)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e < ne) cnt[e] = dblk[ent[e].x].n;
}

// Per tile: first column (colptr) and first element (base) of its stream;
// colptr[nt] closes the last tile.
__global__ void k_tile_streams(const int64_t* __restrict__ ptr, int64_t nt, int64_t ne,
                               const int64_t* __restrict__ ecol, int64_t ncols,
                               const int64_t* __restrict__ eoff, int64_t nelem,
                               int64_t* __restrict__ colptr, int64_t* __restrict__ base)
{
    int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q > nt) return;
    const int64_t e = ptr[q];
    colptr[q] = e < ne ? ecol[e] : ncols;
    if (q < nt) base[q] = e < ne ? eoff[e] : nelem;
}

// Multiplier index of every column: t offset of the block (low rank) or its
// Morton column (dense).
__global__ void k_fill_ucol(const int2* __restrict__ ent, int64_t ne, const int32_t* __restrict__ rank,
                            const int64_t* __restrict__ toff, const int64_t* __restrict__ ecol,
                            int32_t* __restrict__ ucol_t)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    const int b = ent[e].x;
    const int k = rank[b];
    for (int c = 0; c < k; ++c) ucol_t[ecol[e] + c] = (int32_t)(toff[b] + c);
}

__global__ void k_fill_ncol(const int2* __restrict__ ent, int64_t ne, const Blk* __restrict__ dblk,
                            const int64_t* __restrict__ ecol, int32_t* __restrict__ ncol_x)
{
    int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    const Blk B = dblk[ent[e].x];
    for (int c = 0; c < B.n; ++c) ncol_x[ecol[e] + c] = (int32_t)(B.col0 + c);
}

// Gather work items: a tile's U-then-near column stream in pieces of at most
// ITEM_COLS columns, so that the few tiles with very many near-field columns
// (clusters of coincident points are mutually inadmissible) do not leave one
// CTA streaming long after the others have finished.
constexpr int64_t ITEM_COLS = 4096;

// Symmetric low-rank part: class of every admissible block (1: mirror,
// row0 > col0) and, for a canonical block, the index of its mirror (col0,
// row0) in the (row0, col0)-ordered list (-1 when the list lacks it, as in a
// block-row share).
__global__ void k_adm_class(const Blk* __restrict__ blk, int64_t n, int32_t* __restrict__ cls,
                            int32_t* __restrict__ mir)
{
    const int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    const Blk B = blk[b];
    cls[b] = B.row0 > B.col0 ? 1 : 0;
    int32_t m = -1;
    if (B.row0 < B.col0) {
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            const Blk C = blk[mid];
            if (C.row0 < B.col0 || (C.row0 == B.col0 && C.col0 < B.row0)) lo = mid + 1;
            else hi = mid;
        }
        const Blk C = blk[lo];
        if (C.row0 == B.col0 && C.col0 == B.row0) m = (int32_t)lo;
    }
    mir[b] = m;
}

// First mirror column of every tile's U stream (class-1 entries follow the
// class-0 ones within a tile).
// (umid starts as the end of the tile's U stream; the first class-1 entry
// of a tile, the one whose predecessor in the tile is class 0, sets it)
__global__ void k_umid_init(const int64_t* __restrict__ ucol_ptr, int64_t nt,
                            int64_t* __restrict__ umid)
{
    const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q < nt) umid[q] = ucol_ptr[q + 1];
}

__global__ void k_umid(const int64_t* __restrict__ ptr, const int2* __restrict__ ent,
                       const int32_t* __restrict__ et, const int32_t* __restrict__ cls,
                       const int64_t* __restrict__ ecol, int64_t ne, int64_t* __restrict__ umid)
{
    const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= ne || cls[ent[e].x] == 0) return;
    const int32_t q = et[e];
    if (e == ptr[q] || cls[ent[e - 1].x] == 0) umid[q] = ecol[e];
}

// Pass A / pass B columns of every tile (A: canonical U + near; B: mirror U).
__global__ void k_pass_cols(const int64_t* __restrict__ ucol_ptr, const int64_t* __restrict__ umid,
                            const int64_t* __restrict__ ncol_ptr, int64_t nt,
                            int64_t* __restrict__ ca, int64_t* __restrict__ cb)
{
    const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= nt) return;
    ca[q] = (umid[q] - ucol_ptr[q]) + (ncol_ptr[q + 1] - ncol_ptr[q]);
    cb[q] = ucol_ptr[q + 1] - umid[q];
}

// Items over per-tile column counts c[q]: pieces of at most ITEM_COLS
// columns; a tile without columns gets one item when keep_empty.
__global__ void k_items_from_counts(const int64_t* __restrict__ c, int64_t nt, int keep_empty,
                                    int64_t* __restrict__ cnt)
{
    const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q < nt) cnt[q] = c[q] > 0 ? ceil_div(c[q], ITEM_COLS) : (keep_empty ? 1 : 0);
}

__global__ void k_items_emit_counts(const int64_t* __restrict__ c, int64_t nt,
                                    const int64_t* __restrict__ off, int3* __restrict__ items)
{
    const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= nt) return;
    const int64_t n = off[q + 1] - off[q];
    for (int64_t i = 0; i < n; ++i)
        items[off[q] + i] = make_int3((int)q, (int)(i * ITEM_COLS),
                                      (int)(c[q] < (i + 1) * ITEM_COLS ? c[q] : (i + 1) * ITEM_COLS));
}

// Symmetric near field: the near entries of off-diagonal leaves (row0 !=
// col0; the list holds only leaves with row0 <= col0) give transposed
// products over their columns, which are rows of the mirror leaf. zblk[j]
// describes entry j's transposed range as a block whose rows are the
// entry's columns, so that build_csr cuts it into tiles; zcol[j] is the
// near-stream index of the entry's first column.
__global__ void k_z_flag(const int2* __restrict__ ent, int64_t ne, const Blk* __restrict__ dblk,
                         int64_t* __restrict__ f)
{
    const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= ne) return;
    const Blk B = dblk[ent[e].x];
    f[e] = B.row0 != B.col0 ? 1 : 0;
}

__global__ void k_z_blocks(const int2* __restrict__ ent, int64_t ne, const Blk* __restrict__ dblk,
                           const int64_t* __restrict__ f, const int64_t* __restrict__ off,
                           const int64_t* __restrict__ ecol, Blk* __restrict__ zblk,
                           int64_t* __restrict__ zcol)
{
    const int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (e >= ne || !f[e]) return;
    const Blk B = dblk[ent[e].x];
    Blk Z;
    Z.row0 = B.col0;
    Z.col0 = B.row0;
    Z.m = B.n;
    Z.n = 0;
    zblk[off[e]] = Z;
    zcol[off[e]] = ecol[e];
}

// Per record r (transposed range j met by tile q at row offset o of the
// range): the zbuf entry of the tile's first row and the rows it covers.
__global__ void k_z_records(const int2* __restrict__ zent, const int32_t* __restrict__ zt,
                            int64_t nr, const Blk* __restrict__ zblk,
                            const int64_t* __restrict__ zcol, const int32_t* __restrict__ tile_m,
                            int64_t* __restrict__ zbase, int32_t* __restrict__ zlen)
{
    const int64_t r = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (r >= nr) return;
    const int j = zent[r].x, o = zent[r].y;
    zbase[r] = zcol[j] + o;
    zlen[r] = min(tile_m[zt[r]], zblk[j].m - o);
}

// Gather work items: a tile's U-then-near column stream in pieces of at most
// ITEM_COLS columns (defined above).

__global__ void k_item_count(const int64_t* __restrict__ ucol_ptr, const int64_t* __restrict__ ncol_ptr,
                             int64_t nt, int64_t* __restrict__ cnt)
{
    int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= nt) return;
    const int64_t c = (ucol_ptr[q + 1] - ucol_ptr[q]) + (ncol_ptr[q + 1] - ncol_ptr[q]);
    cnt[q] = c > 0 ? ceil_div(c, ITEM_COLS) : 1;
}

__global__ void k_item_emit(const int64_t* __restrict__ ucol_ptr, const int64_t* __restrict__ ncol_ptr,
                            int64_t nt, const int64_t* __restrict__ off, int3* __restrict__ items)
{
    int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= nt) return;
    const int64_t c = (ucol_ptr[q + 1] - ucol_ptr[q]) + (ncol_ptr[q + 1] - ncol_ptr[q]);
    const int64_t k = c > 0 ? ceil_div(c, ITEM_COLS) : 1;
    for (int64_t i = 0; i < k; ++i)
        items[off[q] + i] = make_int3((int)q, (int)(i * ITEM_COLS),
                                       (int)(c < (i + 1) * ITEM_COLS ? c : (i + 1) * ITEM_COLS));
}

}  // namespace

void mvp_build_lists(const Blk* ablk, const int32_t* rank, int64_t n_adm, const Blk* dblk,
                     int64_t n_dense, const int64_t* leaf_row0, const int32_t* leaf_m,
                     int64_t n_tiles, MvpLists& L, cudaStream_t s, int sym_near)
{
    L.n_tiles = n_tiles;
    L.sym_near = sym_near;
    // symmetric low-rank part: class 1 = mirror blocks (row0 > col0), whose
    // slices follow the canonical ones in every tile
    DevBuf<int32_t> acls;
    if (sym_near) {
        acls.alloc(std::max<int64_t>(n_adm, 1), s);
        L.mirror_of.alloc(std::max<int64_t>(n_adm, 1), s);
        if (n_adm > 0) {
            k_adm_class<<<grid_for(n_adm), NT, 0, s>>>(ablk, n_adm, acls.p, L.mirror_of.p); note_launch();
        }
        build_csr(ablk, n_adm, leaf_row0, n_tiles, L.lr_ptr, L.lr_ent, s, acls.p, &L.lr_boff,
                  &L.lr_pos);
    } else {
        build_csr(ablk, n_adm, leaf_row0, n_tiles, L.lr_ptr, L.lr_ent, s);
    }
    build_csr(dblk, n_dense, leaf_row0, n_tiles, L.dn_ptr, L.dn_ent, s);
    {
        int64_t h[2] = {0, 0};
        HM_CUDA(cudaMemcpyAsync(&h[0], L.lr_ptr.p + n_tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(&h[1], L.dn_ptr.p + n_tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        L.n_lr = h[0];
        L.n_dn = h[1];
    }
    L.lr_tile.alloc(std::max<int64_t>(L.n_lr, 1), s);
    L.dn_tile.alloc(std::max<int64_t>(L.n_dn, 1), s);
    if (n_tiles > 0) {
        k_entry_tiles<<<(unsigned)n_tiles, 64, 0, s>>>(L.lr_ptr.p, n_tiles, L.lr_tile.p); note_launch();
        k_entry_tiles<<<(unsigned)n_tiles, 64, 0, s>>>(L.dn_ptr.p, n_tiles, L.dn_tile.p); note_launch();
    }
    // dense slices: offsets and descriptors
    L.dn_desc.alloc(std::max<int64_t>(L.n_dn, 1), s);
    if (L.n_dn > 0) {
        DevBuf<int64_t> sz(L.n_dn, s), off(L.n_dn + 1, s);
        k_dn_sizes<<<grid_for(L.n_dn), NT, 0, s>>>(L.dn_ent.p, L.dn_tile.p, L.n_dn, dblk, leaf_m, sz.p); note_launch();
        scan_exclusive_i64(sz.p, off.p, L.n_dn, off.p + L.n_dn, s);
        k_dn_desc<<<grid_for(L.n_dn), NT, 0, s>>>(L.dn_ent.p, L.n_dn, dblk, off.p, L.dn_desc.p); note_launch();
        HM_CUDA(cudaMemcpyAsync(&L.near_elems, off.p + L.n_dn, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        // the near-field column stream of every tile
        DevBuf<int64_t> cnt(L.n_dn, s), ecol(L.n_dn + 1, s);
        k_dn_ncols<<<grid_for(L.n_dn), NT, 0, s>>>(L.dn_ent.p, L.n_dn, dblk, cnt.p); note_launch();
        scan_exclusive_i64(cnt.p, ecol.p, L.n_dn, ecol.p + L.n_dn, s);
        HM_CUDA(cudaMemcpyAsync(&L.n_ncols, ecol.p + L.n_dn, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        if (L.n_ncols > INT32_MAX || n_tiles <= 0) fail(HM_EOVERFLOW, "near-field column stream");
        L.ncol_ptr.alloc(n_tiles + 1, s);
        L.nbase.alloc(n_tiles, s);
        L.ncol_x.alloc(std::max<int64_t>(L.n_ncols, 1), s);
        k_tile_streams<<<grid_for(n_tiles + 1), NT, 0, s>>>(L.dn_ptr.p, n_tiles, L.n_dn, ecol.p,
                                                             L.n_ncols, off.p, L.near_elems,
                                                             L.ncol_ptr.p, L.nbase.p); note_launch();
        k_fill_ncol<<<grid_for(L.n_dn), NT, 0, s>>>(L.dn_ent.p, L.n_dn, dblk, ecol.p, L.ncol_x.p); note_launch();
        HM_CUDA(cudaStreamSynchronize(s));
        if (sym_near) {
            // transposed-product records of the off-diagonal near entries
            DevBuf<int64_t> f(L.n_dn, s), zo(L.n_dn + 1, s);
            k_z_flag<<<grid_for(L.n_dn), NT, 0, s>>>(L.dn_ent.p, L.n_dn, dblk, f.p); note_launch();
            scan_exclusive_i64(f.p, zo.p, L.n_dn, zo.p + L.n_dn, s);
            int64_t nz = 0;
            HM_CUDA(cudaMemcpyAsync(&nz, zo.p + L.n_dn, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            DevBuf<Blk> zblk(std::max<int64_t>(nz, 1), s);
            DevBuf<int64_t> zcol(std::max<int64_t>(nz, 1), s);
            k_z_blocks<<<grid_for(L.n_dn), NT, 0, s>>>(L.dn_ent.p, L.n_dn, dblk, f.p, zo.p, ecol.p,
                                                       zblk.p, zcol.p); note_launch();
            DevBuf<int2> zent;
            build_csr(zblk.p, nz, leaf_row0, n_tiles, L.zptr, zent, s);
            HM_CUDA(cudaMemcpyAsync(&L.n_zrec, L.zptr.p + n_tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            DevBuf<int32_t> zt(std::max<int64_t>(L.n_zrec, 1), s);
            L.zbase.alloc(std::max<int64_t>(L.n_zrec, 1), s);
            L.zlen.alloc(std::max<int64_t>(L.n_zrec, 1), s);
            if (L.n_zrec > 0) {
                k_entry_tiles<<<(unsigned)n_tiles, 64, 0, s>>>(L.zptr.p, n_tiles, zt.p); note_launch();
                k_z_records<<<grid_for(L.n_zrec), NT, 0, s>>>(zent.p, zt.p, L.n_zrec, zblk.p, zcol.p,
                                                              leaf_m, L.zbase.p, L.zlen.p); note_launch();
            }
            L.n_zcols = L.n_ncols;
            HM_CUDA(cudaStreamSynchronize(s));
        }
    } else {
        L.ncol_ptr.alloc(n_tiles + 1, s);
        L.nbase.alloc(std::max<int64_t>(n_tiles, 1), s);
        L.ncol_x.alloc(1, s);
        HM_CUDA(cudaMemsetAsync(L.ncol_ptr.p, 0, (n_tiles + 1) * sizeof(int64_t), s));
        HM_CUDA(cudaMemsetAsync(L.nbase.p, 0, std::max<int64_t>(n_tiles, 1) * sizeof(int64_t), s));
    }
    if (sym_near && !L.zptr.p) {
        L.zptr.alloc(std::max<int64_t>(n_tiles, 0) + 1, s);
        HM_CUDA(cudaMemsetAsync(L.zptr.p, 0, (std::max<int64_t>(n_tiles, 0) + 1) * sizeof(int64_t), s));
        L.zbase.alloc(1, s);
        L.zlen.alloc(1, s);
    }
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
        k_vitems_count<<<grid_for(n_adm), NT, 0, s>>>(ablk, rank, n_adm, cnt.p, mt.p, ism.p, rk.p,
                                                     sym_near ? acls.p : nullptr); note_launch();
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
    // low-rank slices: offsets and descriptors (t offsets are known now)
    L.lr_desc.alloc(std::max<int64_t>(L.n_lr, 1), s);
    if (L.n_lr > 0) {
        DevBuf<int64_t> sz(L.n_lr, s), off(L.n_lr + 1, s);
        k_lr_sizes<<<grid_for(L.n_lr), NT, 0, s>>>(L.lr_ent.p, L.lr_tile.p, L.n_lr, rank, leaf_m, sz.p); note_launch();
        scan_exclusive_i64(sz.p, off.p, L.n_lr, off.p + L.n_lr, s);
        k_lr_desc<<<grid_for(L.n_lr), NT, 0, s>>>(L.lr_ent.p, L.n_lr, rank, off.p, L.toff.p, L.lr_desc.p); note_launch();
        HM_CUDA(cudaMemcpyAsync(&L.u_elems, off.p + L.n_lr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        // the U column stream of every tile
        DevBuf<int64_t> cnt(L.n_lr, s), ecol(L.n_lr + 1, s);
        k_lr_ncols<<<grid_for(L.n_lr), NT, 0, s>>>(L.lr_ent.p, L.n_lr, rank, cnt.p); note_launch();
        scan_exclusive_i64(cnt.p, ecol.p, L.n_lr, ecol.p + L.n_lr, s);
        HM_CUDA(cudaMemcpyAsync(&L.n_ucols, ecol.p + L.n_lr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        if (L.n_ucols > INT32_MAX || L.t_len > INT32_MAX || n_tiles <= 0)
            fail(HM_EOVERFLOW, "low-rank column stream");
        L.ucol_ptr.alloc(n_tiles + 1, s);
        L.ubase.alloc(n_tiles, s);
        L.ucol_t.alloc(std::max<int64_t>(L.n_ucols, 1), s);
        k_tile_streams<<<grid_for(n_tiles + 1), NT, 0, s>>>(L.lr_ptr.p, n_tiles, L.n_lr, ecol.p,
                                                             L.n_ucols, off.p, L.u_elems,
                                                             L.ucol_ptr.p, L.ubase.p); note_launch();
        k_fill_ucol<<<grid_for(L.n_lr), NT, 0, s>>>(L.lr_ent.p, L.n_lr, rank, L.toff.p, ecol.p,
                                                   L.ucol_t.p); note_launch();
        if (sym_near) {
            L.umid.alloc(n_tiles, s);
            k_umid_init<<<grid_for(n_tiles), NT, 0, s>>>(L.ucol_ptr.p, n_tiles, L.umid.p); note_launch();
            k_umid<<<grid_for(L.n_lr), NT, 0, s>>>(L.lr_ptr.p, L.lr_ent.p, L.lr_tile.p, acls.p,
                                                  ecol.p, L.n_lr, L.umid.p); note_launch();
            // lr_ecol: the first U column of every block-major entry
            L.lr_ecol.alloc(L.n_lr, s);
            k_bm_ecol<<<grid_for(L.n_lr), NT, 0, s>>>(L.lr_pos.p, ecol.p, L.n_lr, L.lr_ecol.p); note_launch();
            // the canonical blocks of more than 8 slices
            DevBuf<int64_t> bf(n_adm, s), bo(n_adm + 1, s);
            k_big_flag<<<grid_for(n_adm), NT, 0, s>>>(L.mirror_of.p, L.lr_boff.p, L.n_lr, n_adm,
                                                     bf.p); note_launch();
            scan_exclusive_i64(bf.p, bo.p, n_adm, bo.p + n_adm, s);
            HM_CUDA(cudaMemcpyAsync(&L.n_big, bo.p + n_adm, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            L.big.alloc(std::max<int64_t>(L.n_big, 1), s);
            k_big_ids<<<grid_for(n_adm), NT, 0, s>>>(bf.p, bo.p, n_adm, L.big.p); note_launch();
        }
        HM_CUDA(cudaStreamSynchronize(s));
    } else {
        L.ucol_ptr.alloc(n_tiles + 1, s);
        L.ubase.alloc(std::max<int64_t>(n_tiles, 1), s);
        L.ucol_t.alloc(1, s);
        HM_CUDA(cudaMemsetAsync(L.ucol_ptr.p, 0, (n_tiles + 1) * sizeof(int64_t), s));
        HM_CUDA(cudaMemsetAsync(L.ubase.p, 0, std::max<int64_t>(n_tiles, 1) * sizeof(int64_t), s));
        if (sym_near) {
            L.umid.alloc(std::max<int64_t>(n_tiles, 1), s);
            HM_CUDA(cudaMemsetAsync(L.umid.p, 0, std::max<int64_t>(n_tiles, 1) * sizeof(int64_t), s));
            L.lr_ecol.alloc(1, s);
        }
    }
    if (sym_near) {
        if (!L.lr_boff.p) L.lr_boff.alloc(1, s);
        if (!L.lr_pos.p) L.lr_pos.alloc(1, s);
        // pass A (canonical U slices, then the near field) and pass B (mirror
        // U slices) work items
        const int64_t nt = std::max<int64_t>(n_tiles, 1);
        DevBuf<int64_t> ca(nt, s), cb(nt, s), cnt(nt, s);
        k_pass_cols<<<grid_for(n_tiles), NT, 0, s>>>(L.ucol_ptr.p, L.umid.p, L.ncol_ptr.p, n_tiles,
                                                     ca.p, cb.p); note_launch();
        L.item_ptr.alloc(nt + 1, s);
        L.item_ptr_b.alloc(nt + 1, s);
        k_items_from_counts<<<grid_for(n_tiles), NT, 0, s>>>(ca.p, n_tiles, 1, cnt.p); note_launch();
        scan_exclusive_i64(cnt.p, L.item_ptr.p, n_tiles, L.item_ptr.p + n_tiles, s);
        k_items_from_counts<<<grid_for(n_tiles), NT, 0, s>>>(cb.p, n_tiles, 0, cnt.p); note_launch();
        scan_exclusive_i64(cnt.p, L.item_ptr_b.p, n_tiles, L.item_ptr_b.p + n_tiles, s);
        HM_CUDA(cudaMemcpyAsync(&L.n_items, L.item_ptr.p + n_tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(&L.n_items_b, L.item_ptr_b.p + n_tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        if (L.n_items + L.n_items_b > INT32_MAX) fail(HM_EOVERFLOW, "too many gather items");
        L.items.alloc(std::max<int64_t>(L.n_items, 1), s);
        L.items_b.alloc(std::max<int64_t>(L.n_items_b, 1), s);
        k_items_emit_counts<<<grid_for(n_tiles), NT, 0, s>>>(ca.p, n_tiles, L.item_ptr.p, L.items.p); note_launch();
        k_items_emit_counts<<<grid_for(n_tiles), NT, 0, s>>>(cb.p, n_tiles, L.item_ptr_b.p, L.items_b.p); note_launch();
        // elements of the canonical slices (the bytes pass A streams)
        std::vector<int64_t> hu(n_tiles + 1), hm(n_tiles);
        std::vector<int32_t> htm(n_tiles);
        if (n_tiles > 0) {
            HM_CUDA(cudaMemcpyAsync(hu.data(), L.ucol_ptr.p, (n_tiles + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaMemcpyAsync(hm.data(), L.umid.p, n_tiles * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaMemcpyAsync(htm.data(), leaf_m, n_tiles * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
        }
        L.u_elems_canon = 0;
        L.n_ucols_canon = 0;
        for (int64_t q = 0; q < n_tiles; ++q) {
            L.u_elems_canon += (hm[q] - hu[q]) * slice_ld(htm[q]);
            L.n_ucols_canon += hm[q] - hu[q];
        }
        HM_LAUNCH("descriptors");
        return;
    }
    // gather work items
    {
        const int64_t nt = std::max<int64_t>(n_tiles, 1);
        DevBuf<int64_t> cnt(nt, s);
        L.item_ptr.alloc(nt + 1, s);
        k_item_count<<<grid_for(n_tiles), NT, 0, s>>>(L.ucol_ptr.p, L.ncol_ptr.p, n_tiles, cnt.p); note_launch();
        scan_exclusive_i64(cnt.p, L.item_ptr.p, n_tiles, L.item_ptr.p + n_tiles, s);
        HM_CUDA(cudaMemcpyAsync(&L.n_items, L.item_ptr.p + n_tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        if (L.n_items > INT32_MAX) fail(HM_EOVERFLOW, "too many gather items");
        L.items.alloc(std::max<int64_t>(L.n_items, 1), s);
        k_item_emit<<<grid_for(n_tiles), NT, 0, s>>>(L.ucol_ptr.p, L.ncol_ptr.p, n_tiles, L.item_ptr.p,
                                                     L.items.p); note_launch();
    }
    HM_LAUNCH("descriptors");
}

void mvp_relayout_u(int precision, const MvpLists& L, const Blk* ablk, const uint64_t* Uptr,
                    const int32_t* tile_m, void* ustore, cudaStream_t s)
{
    if (L.n_lr <= 0) return;
    const unsigned g = (unsigned)ceil_div(L.n_lr * 32, NT);
    if (precision == HM_PREC_FP64)
        k_relayout_u<double><<<g, NT, 0, s>>>(L.lr_ent.p, L.lr_tile.p, L.lr_desc.p, L.n_lr, ablk, Uptr,
                                              tile_m, static_cast<double*>(ustore));
    else
        k_relayout_u<float><<<g, NT, 0, s>>>(L.lr_ent.p, L.lr_tile.p, L.lr_desc.p, L.n_lr, ablk, Uptr,
                                             tile_m, static_cast<float*>(ustore));
    note_launch();
    HM_LAUNCH("relayout U");
}

void mvp_alloc_work(const MvpPlan& P, MvpWork& W, cudaStream_t s)
{
    W.part.alloc(std::max<int64_t>(P.n_items + P.n_items_b, 1) * std::max(P.max_ld, 1), s);
    if (P.sym_near) W.zbuf.alloc(std::max<int64_t>(P.n_ncols, 1), s);
    if (P.umid) W.zubuf.alloc(std::max<int64_t>(P.n_ucols, 1), s);
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

// ---------------------------------------------------------------- tuning
// Launch shapes of the gather kernel: columns in flight per half-warp and
// CTAs per SM. The first product of a kind (precision, near-field format,
// tile leading dimension, log2 of the tile count) on a device times every
// shape once on the real data and keeps the fastest for the process; all
// shapes give bit-identical results.
constexpr int N_TILE_VARIANTS = 5;
// Not a tuned shape of its own: the 128-column bulk-copy kernel for pass B
// of the symmetric product when pass A runs shape 2.
constexpr int TILE_WIDE = 100;

// The bulk-copy variant needs slices of at most 64 rows and 16-byte column
// runs (every format but the single bfloat16 one).
template <class R, int FMT>
int tile_variants(const MvpPlan& P)
{
    return (P.max_ld <= TROWS && FMT != HM_NEAR_BF16) ? 5 : 3;
}

template <class R, int FMT>
void launch_tile(int v, const MvpPlan& P, const R* xm, const R* t, double* part, cudaStream_t s)
{
    const unsigned g = (unsigned)P.n_items;
    if (P.sym_near) {
        // the symmetric near field runs on the bulk-copy kernels only
        // (shape 3: six stages of 64 columns, shape 2: two stages of 128
        // columns, every other shape: four stages of 64 columns)
        if constexpr (sizeof(R) == 4 && FMT != HM_NEAR_BF16) {
            if (P.max_ld > TROWS) fail(HM_ENOTSUP, "symmetric near field: slices above 64 rows");
            const int tcol = v == 2 ? 128 : 64, nst = v == 3 ? 6 : v == 2 ? 2 : 4;
            const int bytes = nst * tcol * col_bytes64<R, FMT>();
            auto kern = v == 2 ? k_tile_tma<R, FMT, 128, 2, true>
                      : nst == 6 ? k_tile_tma<R, FMT, 64, 6, true> : k_tile_tma<R, FMT, 64, 4, true>;
            HM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            kern<<<g, T3_NT, bytes, s>>>(P, xm, t, part);
            note_launch();
            return;
        } else {
            fail(HM_ENOTSUP, "symmetric near field: mixed precision and a paired or FP32 near field");
        }
    }
    if (v == TILE_WIDE) {
        // two stages of 128 columns (pass B of the symmetric product)
        if constexpr (sizeof(R) == 4 && FMT != HM_NEAR_BF16) {
            if (P.max_ld <= TROWS) {
                const int bytes = 2 * 128 * col_bytes64<R, FMT>();
                auto kern = k_tile_tma<R, FMT, 128, 2>;
                HM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
                kern<<<g, T3_NT, bytes, s>>>(P, xm, t, part);
                note_launch();
                return;
            }
        }
        v = 0;
    }
    if (v >= tile_variants<R, FMT>(P)) v = 0;
    switch (v) {
    case 0: k_tile<R, FMT, 8, 3><<<g, TILE_NT, 0, s>>>(P, xm, t, part); break;
    case 1: k_tile<R, FMT, 16, 2><<<g, TILE_NT, 0, s>>>(P, xm, t, part); break;
    case 2: k_tile<R, FMT, 4, 4><<<g, TILE_NT, 0, s>>>(P, xm, t, part); break;
    case 3: {
        const int bytes = 6 * 64 * col_bytes64<R, FMT>();
        auto kern = k_tile_tma<R, FMT, 64, 6>;
        HM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        kern<<<g, T3_NT, bytes, s>>>(P, xm, t, part);
        break;
    }
    default: {
        const int bytes = 4 * 64 * col_bytes64<R, FMT>();
        auto kern = k_tile_tma<R, FMT, 64, 4>;
        HM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        kern<<<g, T3_NT, bytes, s>>>(P, xm, t, part);
        break;
    }
    }
    note_launch();
}

struct TileKey {
    int dev, precision, fmt, ld, lg_tiles, sym;
    bool operator<(const TileKey& o) const
    {
        return std::tie(dev, precision, fmt, ld, lg_tiles, sym) <
               std::tie(o.dev, o.precision, o.fmt, o.ld, o.lg_tiles, o.sym);
    }
};
std::mutex g_tune_mu;
std::map<TileKey, int> g_tune;

TileKey tile_key(const MvpPlan& P)
{
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    int lg = 0;
    while ((1ll << lg) < P.n_tiles) ++lg;
    return TileKey{dev, P.precision, P.near_format, P.max_ld, lg, P.sym_near};
}

std::atomic<int> g_forced_shape{-1};

int tile_variant(const MvpPlan& P)
{
    const int f = g_forced_shape.load();
    if (f >= 0) return f;
    const TileKey k = tile_key(P);
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(k);
    return it == g_tune.end() ? -1 : it->second;
}

template <class R, int FMT>
int tune_tile(const MvpPlan& P, const R* xm, const R* t, double* part, cudaStream_t s)
{
    cudaEvent_t ev[N_TILE_VARIANTS + 1];
    for (auto& e : ev) HM_CUDA(cudaEventCreate(&e));
    // a first untimed run settles caches and clocks; every run writes the
    // same partial sums
    const int nv = tile_variants<R, FMT>(P);
    launch_tile<R, FMT>(0, P, xm, t, part, s);
    HM_CUDA(cudaEventRecord(ev[0], s));
    for (int v = 0; v < nv; ++v) {
        launch_tile<R, FMT>(v, P, xm, t, part, s);
        HM_CUDA(cudaEventRecord(ev[v + 1], s));
    }
    HM_CUDA(cudaEventSynchronize(ev[nv]));
    int best = 0;
    float tbest = 0.f;
    for (int v = 0; v < nv; ++v) {
        float ms = 0.f;
        HM_CUDA(cudaEventElapsedTime(&ms, ev[v], ev[v + 1]));
        if (v == 0 || ms < tbest) {
            tbest = ms;
            best = v;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[tile_key(P)] = best;
    return best;
}

template <class R, int FMT>
void run_typed(const MvpPlan& P, R* xm, R* t, R* tp, double* part, const double* x, double* y,
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
    if (P.n_tiles > 0 && P.umid) {
        // symmetric low-rank part (float plans with the symmetric near
        // field): pass A, the mirror blocks' t, pass B, finish
        if constexpr (sizeof(R) == 4) {
            MvpPlan A = P;
            A.uview = 1;
            int v = tile_variant(A);
            if (v < 0) v = tune_tile<R, FMT>(A, xm, t, part, s);
            launch_tile<R, FMT>(v, A, xm, t, part, s);
            if (rec) HM_CUDA(cudaEventRecord(rec->e[3], s));
            if (P.n_adm > 0) {
                k_tmirror_small<<<grid_for(P.n_adm), NT, 0, s>>>(
                    P.rank, P.mirror_of, P.lr_boff, P.lr_ecol, P.n_lr, P.n_adm, P.toff,
                    P.zubuf, t); note_launch();
                if (P.n_big > 0) {
                    k_tmirror_big<<<(unsigned)ceil_div(P.n_big * 32, NT), NT, 0, s>>>(
                        P.big, P.n_big, P.rank, P.mirror_of, P.lr_boff, P.lr_ecol, P.n_lr,
                        P.n_adm, P.toff, P.zubuf, t); note_launch();
                }
            }
            if (P.n_items_b > 0) {
                MvpPlan B = P;
                B.uview = 2;
                B.sym_near = 0;          // no near field and no transposed products
                B.zubuf = nullptr;
                B.items = P.items_b;
                B.n_items = P.n_items_b;
                launch_tile<R, FMT>(v == 3 ? 3 : v == 2 ? TILE_WIDE : 4, B, xm, t,
                                    part + P.n_items * P.max_ld, s);
            }
            k_tile_finish_sym<<<(unsigned)P.n_tiles, 256, 0, s>>>(P, part, x, y, accumulate);
            note_launch();
        } else {
            fail(HM_ENOTSUP, "symmetric low-rank part: single precision only");
        }
    } else if (P.n_tiles > 0) {
        int v = tile_variant(P);
        if (v < 0) v = tune_tile<R, FMT>(P, xm, t, part, s);
        const int64_t bs = mvp_batch_items();
        if (bs > 0 && bs < P.n_items) {
            // launches of at most bs work items; each item keeps its partial
            // slot, so the sums are those of one launch
            for (int64_t i0 = 0; i0 < P.n_items; i0 += bs) {
                MvpPlan Q = P;
                Q.items = P.items + i0;
                Q.n_items = std::min(bs, P.n_items - i0);
                launch_tile<R, FMT>(v, Q, xm, t, part + i0 * P.max_ld, s);
            }
        } else {
            launch_tile<R, FMT>(v, P, xm, t, part, s);
        }
        if (rec) HM_CUDA(cudaEventRecord(rec->e[3], s));
        if (P.sym_near)
            k_tile_finish_sym<<<(unsigned)P.n_tiles, 256, 0, s>>>(P, part, x, y, accumulate);
        else
            k_tile_finish<<<grid_for(P.n_tiles * 32), NT, 0, s>>>(P, part, x, y, accumulate);
        note_launch();
    }
    if (rec && P.n_tiles <= 0) HM_CUDA(cudaEventRecord(rec->e[3], s));
    if (rec) HM_CUDA(cudaEventRecord(rec->e[4], s));
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
        for (int k = 0; k < 5; ++k) HM_CUDA(cudaEventCreate(&r.e[k]));
    }
    recs.push_back(r);
    return &recs.back();
}

void MvpTimer::collect()
{
    for (Rec& r : recs) {
        HM_CUDA(cudaEventSynchronize(r.e[4]));
        float a = 0, b = 0, c = 0, d = 0;
        HM_CUDA(cudaEventElapsedTime(&a, r.e[0], r.e[1]));
        HM_CUDA(cudaEventElapsedTime(&b, r.e[1], r.e[2]));
        HM_CUDA(cudaEventElapsedTime(&c, r.e[2], r.e[3]));
        HM_CUDA(cudaEventElapsedTime(&d, r.e[3], r.e[4]));
        t_gather += a;
        t_vtx += b;
        t_tile += c;
        t_tail += d;
        t_total += a + b + c + d;
        ++count;
        pool.push_back(r);
    }
    recs.clear();
}

MvpTimer::~MvpTimer()
{
    for (Rec& r : recs) pool.push_back(r);
    for (Rec& r : pool)
        for (int k = 0; k < 5; ++k) cudaEventDestroy(r.e[k]);
}

namespace {

}  // namespace

int mvp_force_shape(int shape)
{
    if (shape < -1 || shape >= N_TILE_VARIANTS) return HM_EINVAL;
    g_forced_shape.store(shape);
    return HM_OK;
}

namespace {
std::atomic<uint64_t> g_wait_ns{2000000000ull};
std::atomic<int> g_withhold{-1};
}  // namespace

uint64_t mvp_wait_ns() { return g_wait_ns.load(); }
int mvp_withhold() { return g_withhold.load(); }
void set_mvp_wait_ns(uint64_t ns) { g_wait_ns = ns ? ns : 2000000000ull; }
void set_mvp_withhold(int k) { g_withhold = k; }

void mvp_run(const MvpPlan& P0, MvpWork& W, const double* x, double* y, int accumulate,
             cudaStream_t s, MvpTimer* timer)
{
    MvpPlan P = P0;
    P.wait_ns = mvp_wait_ns();
    P.withhold = mvp_withhold();
    P.zbuf = W.zbuf.p;
    P.zubuf = P.umid ? W.zubuf.p : nullptr;
    if (P.precision == HM_PREC_FP64) {
        run_typed<double, HM_NEAR_FP64>(P, W.xm64.p, W.t64.p, W.tp64.p, W.part.p, x, y, accumulate, s, timer);
        return;
    }
    switch (P.near_format) {
    case HM_NEAR_FP64:
        run_typed<float, HM_NEAR_FP64>(P, W.xm32.p, W.t32.p, W.tp32.p, W.part.p, x, y, accumulate, s, timer);
        break;
    case HM_NEAR_FP32:
        run_typed<float, HM_NEAR_FP32>(P, W.xm32.p, W.t32.p, W.tp32.p, W.part.p, x, y, accumulate, s, timer);
        break;
    case HM_NEAR_BF16X2:
        run_typed<float, HM_NEAR_BF16X2>(P, W.xm32.p, W.t32.p, W.tp32.p, W.part.p, x, y, accumulate, s, timer);
        break;
    default:
        run_typed<float, HM_NEAR_BF16>(P, W.xm32.p, W.t32.p, W.tp32.p, W.part.p, x, y, accumulate, s, timer);
        break;
    }
}

}  // namespace hm
