// hm_mvp_nr.cu -- the H-matrix product for several right-hand sides at once:
// Alg. 3 (in the batched form of Sec. 5.4) applied to the columns of X. A
// group of up to 16 vectors shares one pass over the stored factors and near
// field, so every stored entry is read once per group instead of once per
// vector; the gather stays bound by HBM while the group is narrow enough for
// the FP32 pipes.
//
// Layout of a group of NRC (8 or 16) vectors, a narrower group padded with
// zero vectors: the permuted right-hand sides are point-major, xm[i*NRC + r];
// so is t, t[(toff_b + l)*NRC + r]; the partial row sums of the gather items
// are part[(item*max_ld + row)*NRC + r] in double.
//
// Summation order, the same for every vector whatever the group width and the
// vector's place in it (the result for one vector does not depend on the
// vectors multiplied with it):
//  - t_b: lane j of a warp sums the columns j, j + 32, ... of a 256-column
//    chunk of V_b in that order with fused multiply-adds; the 32 lane sums
//    meet in the xor-butterfly tree of masks 16, 8, 4, 2, 1; the chunks of a
//    block add in chunk order.
//  - rows of y: column lane j (of four) takes the columns j, j + 4, ... of
//    every 64-column chunk of the item's U stream and then of its near-field
//    stream; the plain FP32 sum of its 16 columns of a chunk goes into a
//    compensated accumulator; the four lane sums add in lane order in double,
//    the items of a tile in item order, then sigma^2 x.
#include "hm_kernel_fn.cuh"
#include "hm_stream.cuh"

namespace hm {

namespace {

constexpr int NT = 256;
constexpr int VN_W = 4;          // warps per CTA of the V^T X kernel
constexpr int TN_COL = 64;       // columns per bulk-copy chunk
constexpr int TN_STAGES = 4;     // chunks in flight per CTA
constexpr int TN_ROWS = 64;      // slices of at most 64 rows
constexpr int TN_LANES = 4;      // column lanes

inline unsigned grid_for(int64_t n, int nt = NT) { return (unsigned)ceil_div(n, nt); }

// xm[i*NRC + r] = x[r*N + perm[i]] for r < nr, zero for the padding.
template <int NRC>
__global__ void k_gather_xn(const double* __restrict__ x, const int64_t* __restrict__ perm,
                            int64_t N, int nr, float* __restrict__ xm)
{
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i >= N) return;
    const int64_t p = perm[i];
    float v[NRC];
#pragma unroll
    for (int r = 0; r < NRC; ++r) v[r] = r < nr ? (float)x[(int64_t)r * N + p] : 0.f;
    float4* o = reinterpret_cast<float4*>(xm + i * NRC);
#pragma unroll
    for (int g = 0; g < NRC / 4; ++g) o[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
}

// Warp totals of v[0 .. NV-1] at once (NV a power of two, at least 32): each
// xor step m = 16, 8, 4, 2, 1 swaps half of the remaining values (a lane
// keeps the half its lane bit m selects). Every addition is one of the
// xor-butterfly tree's, so each total is bit for bit that of a butterfly
// over one value. Afterwards lane q holds in v[0 .. NV/32 - 1] the totals of
// entries (NV/32) q, (NV/32) q + 1, ...
template <int NV>
__device__ __forceinline__ void warp_scatter_sum(float (&v)[NV], int lane)
{
    static_assert(NV >= 32 && (NV & (NV - 1)) == 0, "power of two, at least 32");
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int m = 16 >> st;
        const int h = NV >> (st + 1);
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[h + i];
            const float keep = up ? v[h + i] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
}

constexpr int VN_LB = 4;   // factor columns l per pass of the V^T X kernel

// t partials for NRC vectors: one warp per (block, 256-column chunk) work
// item, its chunk of X staged in shared memory (rows padded to NRC + 4 floats
// so that the 16-byte reads of a quarter warp hit distinct banks). A pass
// takes VN_LB factor columns l at once, so every staged x is read once per
// pass; lane j holds the factor entries of columns j, j + 32, ... of those
// l and loads the next pass's while it multiplies (packed FP32 pairs).
template <int NRC>
__global__ void __launch_bounds__(VN_W * 32, 2)
k_vtx_n(const Blk* __restrict__ blk, const int32_t* __restrict__ rank,
        const uint64_t* __restrict__ Vptr, const int2* __restrict__ items, int64_t nitems,
        const int64_t* __restrict__ dst, const float* __restrict__ xm, float* __restrict__ t,
        float* __restrict__ tp)
{
    constexpr int XS = NRC + 4;
    constexpr int NV = VN_LB * NRC;        // sums per pass
    constexpr int PER = NV / 32;           // totals a lane writes per pass
    extern __shared__ __align__(16) float xsh[];
    const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * VN_W + wi;
    if (w >= nitems) return;   // no CTA-wide barrier follows
    float* xs = xsh + wi * VCH * XS;
    const int2 it = items[w];
    const int b = it.x, c0 = it.y;
    const Blk B = blk[b];
    const int k = rank[b];
    const int n = B.n;
    const int cn = min(VCH, n - c0);
    const float4* src = reinterpret_cast<const float4*>(xm + (int64_t)(B.col0 + c0) * NRC);
    for (int q = lane; q < VCH * (NRC / 4); q += 32) {
        const int c = q / (NRC / 4), g = q % (NRC / 4);
        const float4 v = c < cn ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(xs + c * XS + 4 * g) = v;
    }
    __syncwarp();
    const float* __restrict__ V = reinterpret_cast<const float*>(Vptr[b]);
    const int64_t d = dst[w];
    float* out = d >= 0 ? tp + d * NRC : t + (-d - 1) * NRC;
    float vn[VN_LB][8];
    auto loadv = [&](int l0) {
#pragma unroll
        for (int l = 0; l < VN_LB; ++l) {
            const float* Vl = V + (int64_t)(l0 + l) * n + c0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int jj = lane + 32 * q;
                vn[l][q] = (l0 + l < k && jj < cn) ? __ldcs(Vl + jj) : 0.f;
            }
        }
    };
    if (k > 0) loadv(0);
    for (int l0 = 0; l0 < k; l0 += VN_LB) {
        float vc[VN_LB][8];
#pragma unroll
        for (int l = 0; l < VN_LB; ++l)
#pragma unroll
            for (int q = 0; q < 8; ++q) vc[l][q] = vn[l][q];
        if (l0 + VN_LB < k) loadv(l0 + VN_LB);
        float2 s2[VN_LB][NRC / 2];
#pragma unroll
        for (int l = 0; l < VN_LB; ++l)
#pragma unroll
            for (int r = 0; r < NRC / 2; ++r) s2[l][r] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float* xr = xs + (lane + 32 * q) * XS;
#pragma unroll
            for (int g = 0; g < NRC / 4; ++g) {
                const float4 xv = *reinterpret_cast<const float4*>(xr + 4 * g);
                const float2 x01 = make_float2(xv.x, xv.y), x23 = make_float2(xv.z, xv.w);
#pragma unroll
                for (int l = 0; l < VN_LB; ++l) {
                    const float2 vv = make_float2(vc[l][q], vc[l][q]);
                    s2[l][2 * g] = __ffma2_rn(vv, x01, s2[l][2 * g]);
                    s2[l][2 * g + 1] = __ffma2_rn(vv, x23, s2[l][2 * g + 1]);
                }
            }
        }
        float val[NV];
#pragma unroll
        for (int l = 0; l < VN_LB; ++l)
#pragma unroll
            for (int r = 0; r < NRC / 2; ++r) {
                val[l * NRC + 2 * r] = s2[l][r].x;
                val[l * NRC + 2 * r + 1] = s2[l][r].y;
            }
        warp_scatter_sum<NV>(val, lane);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = PER * lane + i;
            if (l0 + idx / NRC < k) out[(int64_t)l0 * NRC + idx] = val[i];
        }
    }
}

// Sum the chunk partials of blocks that span several chunks (chunk order).
template <int NRC>
__global__ void k_tsum_n(const int32_t* __restrict__ multi, int64_t nmulti,
                         const int32_t* __restrict__ rank, const int32_t* __restrict__ first,
                         const int32_t* __restrict__ count, const int64_t* __restrict__ dst,
                         const int64_t* __restrict__ toff, const float* __restrict__ tp,
                         float* __restrict__ t)
{
    const int64_t q = blockIdx.x;
    if (q >= nmulti) return;
    const int b = multi[q];
    const int k = rank[b];
    const int f = first[b], cnt = count[b];
    for (int e = threadIdx.x; e < k * NRC; e += blockDim.x) {
        const int l = e / NRC, r = e % NRC;
        float s = 0.f;
        for (int c = 0; c < cnt; ++c) s += tp[(dst[f + c] + l) * NRC + r];
        t[(toff[b] + l) * NRC + r] = s;
    }
}

// Bytes of one 64-row column in the near-field store (U columns are float:
// 256 bytes, never more).
template <int FMT>
__host__ __device__ constexpr int ncol_bytes64()
{
    return FMT == HM_NEAR_FP64 ? 512 : 256;
}

__device__ __forceinline__ void consumer_sync(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Exact rounding error of s + v added to the correction (Knuth's TwoSum,
// branch-free, on packed FP32 pairs; a - b is written fma(b, -1, a), which
// rounds once like the subtraction). s + c is the compensated sum.
__device__ __forceinline__ void two_sum_add(float2& s, float2& c, float2 v)
{
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 t = __fadd2_rn(s, v);
    const float2 bp = __ffma2_rn(s, m1, t);    // t - s
    const float2 ap = __ffma2_rn(bp, m1, t);   // t - bp
    const float2 da = __ffma2_rn(ap, m1, s);   // s - ap
    const float2 db = __ffma2_rn(bp, m1, v);   // v - bp
    c = __fadd2_rn(c, __fadd2_rn(da, db));
    s = t;
}

// ---------------------------------------------------------------- tensor cores
// Near-field chunks in bfloat16 pairs run on the tensor cores (mma.sync
// m16n8k16, bfloat16 operands, FP32 accumulation): the chunk's tile rows x 64
// columns, each entry hi + lo, times the chunk's multipliers (64 columns x
// NRC vectors), each split into three bfloat16 terms x = x1 + x2 + x3 (x1 the
// rounding of x, x2 that of x - x1, x3 that of the rest: 24 bits of x). Five
// products hi x1 + hi x2 + hi x3 + lo x1 + lo x2 carry every term above 2^-24
// of the entry times the multiplier; each product of two bfloat16 numbers is
// exact in FP32. Warp w takes the rows 16 (w mod 4) .. + 15 of every vector
// of the group. Only for slices whose row count is a multiple of 8 (a column's
// hi and lo halves then start on 16-byte boundaries, as ldmatrix needs).
constexpr int XT_LD = TN_COL + 8;   // bf16 per row of a multiplier table (144 bytes)

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t (&r)[2])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Three bfloat16 terms of x (round to nearest each time).
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h1, __nv_bfloat16& h2,
                                       __nv_bfloat16& h3)
{
    h1 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h1);
    h2 = __float2bfloat16_rn(r1);
    h3 = __float2bfloat16_rn(r1 - __bfloat162float(h2));
}

// One near-field chunk on the tensor cores: rows 16 mi .. 16 mi + 15 of
// NRC vectors (NT8 = NRC / 8 tiles of 8), accumulated into c[NT8][4].
template <int NRC>
__device__ __forceinline__ void chunk_mma(const unsigned char* st, int colb, int ld, int cnt,
                                          const __nv_bfloat16 (*xt)[NRC][XT_LD], int mi, int lane,
                                          float (&c)[NRC / 8][4])
{
    constexpr int NT8 = NRC / 8;
    const int mat = lane >> 3, rr = lane & 7;
    const int arow = 16 * mi + 8 * (mat & 1);           // this lane's 8-row block
    const uint32_t abase = smem_addr(st) + (uint32_t)(arow * 2);
    const int bn = lane & 7, bk = 8 * ((lane >> 3) & 1);   // lanes 0..15 address B
#pragma unroll
    for (int ks = 0; ks < TN_COL / 16; ++ks) {
        if (16 * ks >= cnt) break;
        const int acol = 16 * ks + rr + 8 * (mat >> 1);
        uint32_t ahi[4], alo[4];
        ldsm_x4_trans(abase + (uint32_t)(acol * colb), ahi);
        ldsm_x4_trans(abase + (uint32_t)(acol * colb + 2 * ld), alo);
#pragma unroll
        for (int nt = 0; nt < NT8; ++nt) {
            uint32_t b[3][2];
#pragma unroll
            for (int q = 0; q < 3; ++q)
                ldsm_x2(smem_addr(&xt[q][8 * nt + bn][16 * ks + bk]), b[q]);
            mma_bf16(c[nt], ahi, b[0]);
            mma_bf16(c[nt], ahi, b[1]);
            mma_bf16(c[nt], ahi, b[2]);
            mma_bf16(c[nt], alo, b[0]);
            mma_bf16(c[nt], alo, b[1]);
        }
    }
}

// Rows ir .. ir+3 of chunk column col as two packed row pairs.
template <int FMT, bool ISU>
__device__ __forceinline__ void stage_rows(const unsigned char* st, int col, int colb, int ir, int ld,
                                           float2& a01, float2& a23)
{
    if (ISU || FMT == HM_NEAR_FP32) {
        const float4 v = *reinterpret_cast<const float4*>(st + col * colb + 4 * ir);
        a01 = make_float2(v.x, v.y);
        a23 = make_float2(v.z, v.w);
    } else if (FMT == HM_NEAR_BF16X2) {
        const __nv_bfloat16* q = reinterpret_cast<const __nv_bfloat16*>(st + col * colb) + ir;
        const uint2 h = *reinterpret_cast<const uint2*>(q);
        const uint2 l = *reinterpret_cast<const uint2*>(q + ld);
        a01 = __fadd2_rn(bf2(h.x), bf2(l.x));
        a23 = __fadd2_rn(bf2(h.y), bf2(l.y));
    } else {
        const double2* q = reinterpret_cast<const double2*>(st + col * colb + 8 * ir);
        const double2 v0 = q[0], v1 = q[1];
        a01 = make_float2((float)v0.x, (float)v0.y);
        a23 = make_float2((float)v1.x, (float)v1.y);
    }
}

// Plain sums over one thread's columns j, j + 4, ... of a chunk (ascending),
// rows ir .. ir+3 against vectors 4g .. 4g+3; the multiplier table holds
// every multiplier twice ({m0, m0, m1, m1, m2, m2, m3, m3} per column and group).
template <int FMT, bool ISU, bool TAIL, int NRC>
__device__ __forceinline__ void chunk_sums(const unsigned char* st, const float* ms, int j, int ir,
                                           int g, int ld, int colb, int cnt, float2 (&sg)[2][4])
{
#pragma unroll 4
    for (int e = 0; e < TN_COL / TN_LANES; ++e) {
        const int col = j + TN_LANES * e;
        if (TAIL && col >= cnt) break;
        float2 a01, a23;
        stage_rows<FMT, ISU>(st, col, colb, ir, ld, a01, a23);
        const float4* mp = reinterpret_cast<const float4*>(ms + 2 * (col * NRC + 4 * g));
        const float4 mA = mp[0], mB = mp[1];
        const float2 m[4] = {make_float2(mA.x, mA.y), make_float2(mA.z, mA.w),
                             make_float2(mB.x, mB.y), make_float2(mB.z, mB.w)};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            sg[0][r] = __ffma2_rn(a01, m[r], sg[0][r]);
            sg[1][r] = __ffma2_rn(a23, m[r], sg[1][r]);
        }
    }
}

// One CTA per gather work item (a piece of one row tile's U-then-near column
// stream, as in the one-vector product). A producer thread moves 64-column
// chunks into a ring of shared-memory stages with cp.async.bulk; NRC / 2
// consumer warps multiply them. Consumer thread (j, g, q) owns rows
// 4q .. 4q+3, vectors 4g .. 4g+3 and the chunk columns j, j + 4, ..., and
// fetches one float4 of the next chunk's multipliers (column, vector group)
// into a double-buffered table; a named barrier over the consumers publishes
// it. Sums run on packed FP32 pairs (two rows of one vector).
// Waits are bounded: a wait that gives up sets bit 4 of the status word, the
// consumers leave together after their barrier, and the item writes nothing.
template <int FMT, int NRC>
__global__ void __launch_bounds__((NRC / 2 + 1) * 32, 2)
k_tile_n(MvpPlan P, const float* __restrict__ xm, const float* __restrict__ t,
         double* __restrict__ part)
{
    constexpr int NCW = NRC / 2;        // consumer warps
    constexpr int NG = NRC / 4;         // vector groups of four
    constexpr int STAGE = TN_COL * ncol_bytes64<FMT>();
    static_assert(16 * NG * TN_LANES == NCW * 32, "one consumer per (rows, group, lane)");
    static_assert(TN_COL * NG == NCW * 32, "one multiplier float4 per consumer");
    static_assert((TN_LANES + 1) * TN_ROWS * NRC * 8 <= TN_STAGES * STAGE, "row sums fit the stages");
    constexpr int NT8 = NRC / 8;
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ uint64_t full[TN_STAGES], empty[TN_STAGES];
    __shared__ __align__(16) float msm[2][2 * TN_COL * NRC];
    // the tensor cores' multiplier tables (three bfloat16 terms per value)
    __shared__ __align__(16) __nv_bfloat16 xt[FMT == HM_NEAR_BF16X2 ? 2 : 1][3][NRC][XT_LD];
    __shared__ int failed;
    const int64_t item = blockIdx.x;
    const int3 it = P.items[item];
    const int64_t tile = it.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = P.tile_m[tile];
    const int ld = slice_ld(mt);
    const int64_t uc0 = P.ucol_ptr[tile], nu = P.ucol_ptr[tile + 1] - uc0, ub = P.ubase[tile];
    const int64_t nc0 = P.ncol_ptr[tile], nb = P.nbase[tile];
    const int64_t ucb = it.y < nu ? it.y : nu, uce = it.z < nu ? it.z : nu;
    const int64_t ncb = it.y > nu ? it.y - nu : 0, nce = it.z > nu ? it.z - nu : 0;
    const int nuch = (int)ceil_div(uce - ucb, TN_COL), nnch = (int)ceil_div(nce - ncb, TN_COL);
    const int nch = nuch + nnch;
    const int ucolb = ld * 4;
    const int ncolb = FMT == HM_NEAR_FP64 ? ld * 8 : ld * 4;
    // near-field chunks on the tensor cores (bfloat16 pairs, slices of a
    // multiple of 8 rows)
    const bool tc = FMT == HM_NEAR_BF16X2 && (ld & 7) == 0;
    if (tc) {
        // a tensor-core chunk of fewer than 64 columns reads whole 16-column
        // steps, and its columns past the chunk multiply zero multipliers:
        // start from zeroed stages so that they hold finite values (later
        // only earlier chunks' entries); the fence orders these writes before
        // the bulk copies into the same memory
        uint4* z = reinterpret_cast<uint4*>(tsm);
        for (int e = threadIdx.x; e < TN_STAGES * STAGE / 16; e += blockDim.x)
            z[e] = make_uint4(0u, 0u, 0u, 0u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < TN_STAGES; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], NCW);
        }
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto chunk = [&](int k, bool& isu, int64_t& c0, int& cnt) {
        isu = k < nuch;
        c0 = isu ? ucb + (int64_t)k * TN_COL : ncb + (int64_t)(k - nuch) * TN_COL;
        const int64_t cend = isu ? uce : nce;
        cnt = (int)(cend - c0 < TN_COL ? cend - c0 : TN_COL);
    };
    // the four column lanes' row sums, once the stages are no longer read
    double (*ps)[TN_ROWS][NRC] = reinterpret_cast<double (*)[TN_ROWS][NRC]>(tsm);
    if (w == NCW) {
        // ---------------- producer
        if (lane == 0) {
            int k = 0;
            for (; k < nch; ++k) {
                const int slot = k % TN_STAGES;
                if (k >= TN_STAGES && !mbar_wait(&empty[slot], ((k / TN_STAGES) - 1) & 1, P.wait_ns)) {
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
                    ? reinterpret_cast<const char*>(static_cast<const float*>(P.ustore) + ub + c0 * ld)
                    : static_cast<const char*>(P.near) + (int64_t)ncolb * c0 +
                          (FMT == HM_NEAR_FP64 ? 8 * nb : 4 * nb);
                mbar_arrive_tx(&full[slot], bytes);
                bulk_copy(tsm + slot * STAGE, src, bytes, &full[slot]);
            }
            // every copy issued lands before the CTA exits (see k_tile_tma)
            for (int q = (k > TN_STAGES ? k - TN_STAGES : 0); q < k; ++q)
                if (q != P.withhold &&
                    !mbar_wait(&full[q % TN_STAGES], (q / TN_STAGES) & 1, P.wait_ns > MBAR_DRAIN_NS ? P.wait_ns : MBAR_DRAIN_NS))
                    atomicOr(P.status, 4);
        }
    } else {
        // ---------------- consumers
        const int tc_id = threadIdx.x;
        const int rq = tc_id & 15, g = (tc_id >> 4) % NG, j = tc_id / (16 * NG);
        const int ir = 4 * rq;
        const bool act = ir < ld;
        const int fc = tc_id / NG, fg = tc_id % NG;   // the multiplier float4 this thread fetches
        const float4* __restrict__ t4 = reinterpret_cast<const float4*>(t);
        const float4* __restrict__ x4 = reinterpret_cast<const float4*>(xm);
        auto fetch = [&](int k) -> float4 {
            float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k >= nch) return z;
            bool isu;
            int64_t c0;
            int cnt;
            chunk(k, isu, c0, cnt);
            if (fc >= cnt) return z;
            return isu ? t4[(int64_t)P.ucol_t[uc0 + c0 + fc] * NG + fg]
                       : x4[(int64_t)P.ncol_x[nc0 + c0 + fc] * NG + fg];
        };
        // the next chunk's multipliers: a near chunk on the tensor cores
        // takes them split into bfloat16 terms, any other chunk duplicated
        // for the packed FP32 pairs
        auto publish = [&](int buf, float4 m, int kn) {
            if (FMT == HM_NEAR_BF16X2 && tc && kn >= nuch) {
                const float v[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    __nv_bfloat16 h1, h2, h3;
                    split3(v[e], h1, h2, h3);
                    xt[buf & (FMT == HM_NEAR_BF16X2 ? 1 : 0)][0][4 * fg + e][fc] = h1;
                    xt[buf & (FMT == HM_NEAR_BF16X2 ? 1 : 0)][1][4 * fg + e][fc] = h2;
                    xt[buf & (FMT == HM_NEAR_BF16X2 ? 1 : 0)][2][4 * fg + e][fc] = h3;
                }
                return;
            }
            float4* d = reinterpret_cast<float4*>(msm[buf]) + 2 * tc_id;
            d[0] = make_float4(m.x, m.x, m.y, m.y);
            d[1] = make_float4(m.z, m.z, m.w, m.w);
        };
        float tsum[NT8][4], tcmp[NT8][4];   // tensor-core rows: compensated sums
#pragma unroll
        for (int nt = 0; nt < NT8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) tsum[nt][e] = tcmp[nt][e] = 0.f;
        float2 as[2][4], ac[2][4];   // compensated sums and corrections [row pair][vector]
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int r = 0; r < 4; ++r) as[p][r] = ac[p][r] = make_float2(0.f, 0.f);
        float4 mf = fetch(0);
        publish(0, mf, 0);
        consumer_sync(NCW * 32);
        for (int k = 0; k < nch; ++k) {
            const int slot = k % TN_STAGES;
            mf = fetch(k + 1);
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[slot], (k / TN_STAGES) & 1, P.wait_ns));
            bool isu_k;
            {
                int64_t c0k;
                int cntk;
                chunk(k, isu_k, c0k, cntk);
                if (ok && tc && !isu_k) {
                    // a near chunk on the tensor cores: warp w < 4 takes rows
                    // 16 w .. 16 w + 15 of every vector
                    if (w < 4 && 16 * w < ld) {
                        float cz[NT8][4];
#pragma unroll
                        for (int nt = 0; nt < NT8; ++nt)
#pragma unroll
                            for (int e = 0; e < 4; ++e) cz[nt][e] = 0.f;
                        chunk_mma<NRC>(tsm + slot * STAGE, ncolb, ld, cntk,
                                       xt[k & (FMT == HM_NEAR_BF16X2 ? 1 : 0)], w, lane, cz);
#pragma unroll
                        for (int nt = 0; nt < NT8; ++nt) {
                            float2 s01 = make_float2(tsum[nt][0], tsum[nt][1]);
                            float2 c01 = make_float2(tcmp[nt][0], tcmp[nt][1]);
                            float2 s23 = make_float2(tsum[nt][2], tsum[nt][3]);
                            float2 c23 = make_float2(tcmp[nt][2], tcmp[nt][3]);
                            two_sum_add(s01, c01, make_float2(cz[nt][0], cz[nt][1]));
                            two_sum_add(s23, c23, make_float2(cz[nt][2], cz[nt][3]));
                            tsum[nt][0] = s01.x; tsum[nt][1] = s01.y;
                            tsum[nt][2] = s23.x; tsum[nt][3] = s23.y;
                            tcmp[nt][0] = c01.x; tcmp[nt][1] = c01.y;
                            tcmp[nt][2] = c23.x; tcmp[nt][3] = c23.y;
                        }
                    }
                }
            }
            if (ok) {
                if (act && !(tc && !isu_k)) {
                    bool isu;
                    int64_t c0;
                    int cnt;
                    chunk(k, isu, c0, cnt);
                    const unsigned char* st = tsm + slot * STAGE;
                    const float* ms = msm[k & 1];
                    float2 sg[2][4];
#pragma unroll
                    for (int p = 0; p < 2; ++p)
#pragma unroll
                        for (int r = 0; r < 4; ++r) sg[p][r] = make_float2(0.f, 0.f);
                    if (isu) {
                        if (cnt == TN_COL) chunk_sums<FMT, true, false, NRC>(st, ms, j, ir, g, ld, ucolb, cnt, sg);
                        else chunk_sums<FMT, true, true, NRC>(st, ms, j, ir, g, ld, ucolb, cnt, sg);
                    } else {
                        if (cnt == TN_COL) chunk_sums<FMT, false, false, NRC>(st, ms, j, ir, g, ld, ncolb, cnt, sg);
                        else chunk_sums<FMT, false, true, NRC>(st, ms, j, ir, g, ld, ncolb, cnt, sg);
                    }
#pragma unroll
                    for (int p = 0; p < 2; ++p)
#pragma unroll
                        for (int r = 0; r < 4; ++r) two_sum_add(as[p][r], ac[p][r], sg[p][r]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
            } else if (lane == 0) {
                atomicOr(P.status, 4);
                failed = 1;
            }
            publish((k + 1) & 1, mf, k + 1);
            consumer_sync(NCW * 32);
            if (*(volatile int*)&failed) break;
        }
        // every consumer has passed its last barrier, so no stage is read
        // any more (the stages are only reused when nothing failed)
        if (!*(volatile int*)&failed) {
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    ps[j][ir + 2 * p][4 * g + r] =
                        act ? (double)as[p][r].x + (double)ac[p][r].x : 0.0;
                    ps[j][ir + 2 * p + 1][4 * g + r] =
                        act ? (double)as[p][r].y + (double)ac[p][r].y : 0.0;
                }
            // the tensor cores' rows in a fifth slot (zero without them):
            // fragment element e of tile nt is row 16 w + lane / 4 (+ 8 for
            // e >= 2), vector 8 nt + 2 (lane mod 4) (+ 1 for odd e)
            if (w < 4) {
#pragma unroll
                for (int nt = 0; nt < NT8; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        ps[TN_LANES][16 * w + (lane >> 2) + 8 * (e >> 1)][8 * nt + 2 * (lane & 3) + (e & 1)] =
                            (double)tsum[nt][e] + (double)tcmp[nt][e];
            }
        }
    }
    __syncthreads();
    if (*(volatile int*)&failed) return;
    for (int e = threadIdx.x; e < mt * NRC; e += blockDim.x) {
        const int row = e / NRC, r = e % NRC;
        double sum = 0.0;
#pragma unroll
        for (int q = 0; q <= TN_LANES; ++q) sum += ps[q][row][r];
        part[(item * P.max_ld + row) * NRC + r] = sum;
    }
}

// y for every row of every tile and vector: the tile's item sums in item
// order plus sigma^2 x, in the caller's order (one warp per tile).
template <int NRC>
__global__ void k_finish_n(MvpPlan P, const double* __restrict__ part, const double* __restrict__ x,
                           double* __restrict__ y, int nr, int accumulate)
{
    const int64_t tile = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (tile >= P.n_tiles) return;
    const int64_t N = P.Ntot;
    const int64_t r0 = P.tile_row0[tile];
    const int mt = P.tile_m[tile];
    const int64_t i0 = P.item_ptr[tile], i1 = P.item_ptr[tile + 1];
    for (int e = lane; e < mt * NRC; e += 32) {
        const int i = e / NRC, r = e % NRC;
        if (r >= nr) continue;
        double sum = 0.0;
        for (int64_t q = i0; q < i1; ++q) sum += part[(q * P.max_ld + i) * NRC + r];
        const int64_t row = r0 + i;
        const int64_t dst = P.perm[row] + (int64_t)r * N;
        const double sg = P.sig_row ? P.sig_row[row] : P.sigma2;
        const double v = sum + sg * x[dst];
        y[dst] = accumulate ? y[dst] + v : v;
    }
}

template <int FMT, int NRC>
void run_group(const MvpPlan& P, MvpWork& W, const double* x, double* y, int nr, int accumulate,
               cudaStream_t s)
{
    k_gather_xn<NRC><<<grid_for(P.Ntot), NT, 0, s>>>(x, P.perm, P.Ntot, nr, W.xmn.p);
    note_launch();
    if (P.n_vitems > 0) {
        const int smem = VN_W * VCH * (NRC + 4) * (int)sizeof(float);
        auto kv = k_vtx_n<NRC>;
        HM_CUDA(cudaFuncSetAttribute(kv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        kv<<<(unsigned)ceil_div(P.n_vitems, VN_W), VN_W * 32, smem, s>>>(
            P.ablk, P.rank, P.Vptr, P.vitems, P.n_vitems, P.tpart_off, W.xmn.p, W.tn.p, W.tpn.p);
        note_launch();
    }
    if (P.n_multi > 0) {
        k_tsum_n<NRC><<<(unsigned)P.n_multi, 128, 0, s>>>(P.multi, P.n_multi, P.rank, P.tsum_first,
                                                         P.tsum_count, P.tpart_off, P.toff, W.tpn.p,
                                                         W.tn.p);
        note_launch();
    }
    if (P.n_tiles > 0) {
        // (+256 bytes: a tensor-core fragment of the last stage may read up
        // to 16 bytes past it, into this padding)
        const int smem = TN_STAGES * TN_COL * ncol_bytes64<FMT>() + 256;
        auto kt = k_tile_n<FMT, NRC>;
        HM_CUDA(cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        kt<<<(unsigned)P.n_items, (NRC / 2 + 1) * 32, smem, s>>>(P, W.xmn.p, W.tn.p, W.partn.p);
        note_launch();
        k_finish_n<NRC><<<grid_for(P.n_tiles * 32), NT, 0, s>>>(P, W.partn.p, x, y, nr, accumulate);
        note_launch();
    }
    HM_LAUNCH("matvec (several vectors)");
}

template <int NRC>
void run_group_fmt(const MvpPlan& P, MvpWork& W, const double* x, double* y, int nr,
                   int accumulate, cudaStream_t s)
{
    switch (P.near_format) {
    case HM_NEAR_FP64: run_group<HM_NEAR_FP64, NRC>(P, W, x, y, nr, accumulate, s); break;
    case HM_NEAR_FP32: run_group<HM_NEAR_FP32, NRC>(P, W, x, y, nr, accumulate, s); break;
    default: run_group<HM_NEAR_BF16X2, NRC>(P, W, x, y, nr, accumulate, s); break;
    }
}

}  // namespace

bool mvp_multi_fused(const MvpPlan& P)
{
    return P.precision != HM_PREC_FP64 && P.max_ld <= TN_ROWS && !P.sym_near &&
           (P.near_format == HM_NEAR_FP64 || P.near_format == HM_NEAR_FP32 ||
            P.near_format == HM_NEAR_BF16X2);
}

void mvp_run_multi(const MvpPlan& P0, MvpWork& W, const double* x, double* y, int nrhs,
                   int accumulate, cudaStream_t s)
{
    MvpPlan P = P0;
    P.wait_ns = mvp_wait_ns();
    P.withhold = mvp_withhold();
    const int64_t N = P.Ntot;
    if (!mvp_multi_fused(P)) {
        for (int r = 0; r < nrhs; ++r)
            mvp_run(P, W, x + (int64_t)r * N, y + (int64_t)r * N, accumulate, s, nullptr);
        return;
    }
    constexpr int G = MVP_NRC_MAX;
    if (!W.xmn.p) {
        W.xmn.alloc(std::max<int64_t>(N, 1) * G, s);
        W.tn.alloc(std::max<int64_t>(P.t_len, 1) * G, s);
        W.tpn.alloc(std::max<int64_t>(P.tpart_len, 1) * G, s);
        W.partn.alloc(std::max<int64_t>(P.n_items, 1) * std::max(P.max_ld, 1) * G, s);
    }
    for (int c = 0; c < nrhs; c += G) {
        const int nr = std::min(G, nrhs - c);
        const double* xc = x + (int64_t)c * N;
        double* yc = y + (int64_t)c * N;
        if (nr <= 8) run_group_fmt<8>(P, W, xc, yc, nr, accumulate, s);
        else run_group_fmt<16>(P, W, xc, yc, nr, accumulate, s);
    }
}

}  // namespace hm
