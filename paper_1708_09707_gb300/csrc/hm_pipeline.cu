// hm_pipeline.cu -- the build pipeline behind hm_build / hm_build_batch, the
// product driver, exports and conjugate gradients.
//
// Build (Sec. 5): per point set, Morton sort + cluster tree + traversal
// (hm_build.cu); then, over the leaves of all sets at once, block descriptors,
// batched ACA of the admissible leaves (hm_aca.cu), batched evaluation of the
// dense leaves (hm_near.cu) and the gather lists of the product (hm_mvp.cu).
//
// Factor storage. The plain method does not know the ranks before ACA runs,
// so blocks are compressed in passes: each pass reserves min(k_cap, m, n)
// columns per block in a bounded scratch area, runs ACA, then copies the
// rank-k columns into an exactly sized segment. With the learned rank model,
// every block reserves its predicted rank directly in the final store (one
// pass, no copy) and only blocks whose prediction was too small are re-run
// with the full cap.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "hm_handle.cuh"
#include "hm_mlp.cuh"

hm_handle_s::~hm_handle_s()
{
    if (stream) cudaStreamSynchronize(stream);
}

namespace hm {

namespace {

constexpr int NT = 256;
inline unsigned grid_for(int64_t n) { return (unsigned)ceil_div(n, NT); }

int bits_for(int64_t n)
{
    int b = 0;
    while ((1ll << b) < n) ++b;
    return b;
}

// Block descriptors of leaf pairs: tau in the row tree (lo, hi; its set's
// first row row0), sigma in the column tree (lo2, hi2; col0).
__global__ void k_make_blk(const int2* __restrict__ pairs, int64_t n,
                           const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                           int64_t row0, const int32_t* __restrict__ lo2,
                           const int32_t* __restrict__ hi2, int64_t col0, Blk* __restrict__ out)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    int2 p = pairs[b];
    Blk B;
    B.row0 = row0 + lo[p.x];
    B.col0 = col0 + lo2[p.y];
    B.m = hi[p.x] - lo[p.x];
    B.n = hi2[p.y] - lo2[p.y];
    out[b] = B;
}

__global__ void k_leaf_flags(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                             int64_t nn, int C, int64_t* __restrict__ flag)
{
    int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (v >= nn) return;
    flag[v] = (lo[v] >= 0 && hi[v] - lo[v] <= C) ? 1 : 0;
}

__global__ void k_leaf_emit(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                            int64_t nn, const int64_t* __restrict__ flag,
                            const int64_t* __restrict__ off, uint64_t* __restrict__ key,
                            uint32_t* __restrict__ val, int32_t* __restrict__ vid)
{
    int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (v >= nn || !flag[v]) return;
    int64_t o = off[v];
    key[o] = (uint64_t)lo[v];
    val[o] = (uint32_t)o;
    vid[o] = (int32_t)v;
}

__global__ void k_leaf_tiles(const uint32_t* __restrict__ val, const int32_t* __restrict__ vid,
                             int64_t nt, const int32_t* __restrict__ lo,
                             const int32_t* __restrict__ hi, int64_t row0,
                             int64_t* __restrict__ trow, int32_t* __restrict__ tm)
{
    int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= nt) return;
    int v = vid[val[q]];
    trow[q] = row0 + lo[v];
    tm[q] = hi[v] - lo[v];
}

__global__ void k_classes(const Blk* __restrict__ blk, const uint32_t* __restrict__ ids,
                          int64_t n, int kcap, const int32_t* __restrict__ kpred,
                          uint64_t* __restrict__ key, uint32_t* __restrict__ val,
                          int32_t* __restrict__ kres, int64_t* __restrict__ cls_count)
{
    int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= n) return;
    const uint32_t b = ids ? ids[q] : (uint32_t)q;
    Blk B = blk[b];
    int c = aca_class_of(B.m, B.n);
    const int k = aca_reservation(B.m, B.n, kcap, kpred, b);
    kres[b] = k;
    const int kb = aca_kbucket(k);
    // largest class first, then the rank buckets in increasing order
    key[q] = (uint64_t)((ACA_NCLASS - 1 - c) * ACA_NKB + kb);
    val[q] = b;
    atomicAdd((unsigned long long*)&cls_count[c * ACA_NKB + kb], 1ull);
}

// Block-row share (hm_options.row_lo / row_hi): leaf (tau, sigma) stays when
// tau meets the rows [r0, r1), or, in symmetric mode, when it is canonical
// (tau.lo <= sigma.lo) and sigma meets them (the partner of a kept mirror
// leaf).
__global__ void k_row_keep(const int2* __restrict__ pairs, int64_t n,
                           const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                           int64_t r0, int64_t r1, int sym, int64_t* __restrict__ keep)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    const int2 p = pairs[b];
    const bool rows = lo[p.x] < r1 && hi[p.x] > r0;
    const bool partner = sym && lo[p.x] <= lo[p.y] && lo[p.y] < r1 && hi[p.y] > r0;
    keep[b] = (rows || partner) ? 1 : 0;
}

__global__ void k_row_compact(const int2* __restrict__ in, int64_t n,
                              const int64_t* __restrict__ keep, const int64_t* __restrict__ off,
                              int2* __restrict__ out)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b < n && keep[b]) out[off[b]] = in[b];
}

// Keep the leaves of a block-row share, in their canonical order.
int64_t row_filter(DevBuf<int2>& pairs, int64_t n, const int32_t* lo, const int32_t* hi,
                   int64_t r0, int64_t r1, int sym, cudaStream_t s)
{
    if (n == 0) return 0;
    DevBuf<int64_t> keep(n, s), off(n + 1, s);
    k_row_keep<<<grid_for(n), NT, 0, s>>>(pairs.p, n, lo, hi, r0, r1, sym, keep.p); note_launch();
    scan_exclusive_i64(keep.p, off.p, n, off.p + n, s);
    int64_t cnt = 0;
    HM_CUDA(cudaMemcpyAsync(&cnt, off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    DevBuf<int2> out(std::max<int64_t>(cnt, 1), s);
    k_row_compact<<<grid_for(n), NT, 0, s>>>(pairs.p, n, keep.p, off.p, out.p); note_launch();
    HM_LAUNCH("row share");
    pairs = std::move(out);
    return cnt;
}

// Symmetric kernels: leaf b is canonical when its rows start no later than
// its columns; the others are mirrors of a canonical leaf, marked in flags
// (no ACA of their own, no reservation; they still count in the product).
constexpr int MIRROR_FLAG = 4;
__global__ void k_canon_flag(const Blk* __restrict__ blk, int64_t n, int64_t* __restrict__ f)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b < n) f[b] = blk[b].row0 <= blk[b].col0 ? 1 : 0;
}

__global__ void k_canon_ids(const int64_t* __restrict__ f, const int64_t* __restrict__ off, int64_t n,
                            uint32_t* __restrict__ ids)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b < n && f[b]) ids[off[b]] = (uint32_t)b;
}

__global__ void k_canon_blocks(const Blk* __restrict__ blk, const int64_t* __restrict__ f,
                               const int64_t* __restrict__ off, int64_t n, Blk* __restrict__ out)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b < n && f[b]) out[off[b]] = blk[b];
}

// A mirror leaf (sigma, tau) takes the factors of (tau, sigma) with U and V
// exchanged. The leaves are in (row0, col0) order, so its partner is found by
// binary search; a missing partner (not possible for a symmetric block tree)
// sets the status word.
__global__ void k_mirror(const Blk* __restrict__ blk, int64_t n, uint64_t* __restrict__ Uptr,
                         uint64_t* __restrict__ Vptr, int32_t* __restrict__ rank,
                         int32_t* __restrict__ nrej, int32_t* __restrict__ flags, int* status)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    const Blk B = blk[b];
    if (B.row0 <= B.col0) return;
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const Blk M = blk[mid];
        if (M.row0 < B.col0 || (M.row0 == B.col0 && M.col0 < B.row0)) lo = mid + 1;
        else hi = mid;
    }
    const Blk M = blk[lo];
    if (M.row0 != B.col0 || M.col0 != B.row0) {
        atomicOr(status, 8);
        return;
    }
    Uptr[b] = Vptr[lo];
    Vptr[b] = Uptr[lo];
    rank[b] = rank[lo];
    nrej[b] = 0;
    flags[b] = MIRROR_FLAG;
}

// The canonical partner of every admissible leaf: itself when row0 <= col0,
// else the leaf (tau, sigma) of the mirror leaf (sigma, tau), found by binary
// search as in k_mirror; -1 (and the status word) if missing.
__global__ void k_np_partner(const Blk* __restrict__ blk, int64_t n, int64_t* __restrict__ partner,
                             int* status)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    const Blk B = blk[b];
    if (B.row0 <= B.col0) {
        partner[b] = b;
        return;
    }
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const Blk M = blk[mid];
        if (M.row0 < B.col0 || (M.row0 == B.col0 && M.col0 < B.row0)) lo = mid + 1;
        else hi = mid;
    }
    const Blk M = blk[lo];
    if (M.row0 != B.col0 || M.col0 != B.row0) {
        atomicOr(status, 8);
        partner[b] = -1;
        return;
    }
    partner[b] = lo;
}

// Reserved entries of block order[q]: total kres (m + n) and the U part kres m.
__global__ void k_reserve(const Blk* __restrict__ blk, const uint32_t* __restrict__ order,
                          int64_t n, const int32_t* __restrict__ kres, int64_t* __restrict__ res,
                          int64_t* __restrict__ resu)
{
    int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= n) return;
    uint32_t b = order[q];
    res[q] = (int64_t)kres[b] * (blk[b].m + blk[b].n);
    resu[q] = (int64_t)kres[b] * blk[b].m;
}

// U of order[q] at ubase + (preu[q] - preu[q0]), V at vbase + (prev[q] - prev[q0])
// where prev = pre - preu.
__global__ void k_set_ptrs(const uint32_t* __restrict__ order, int64_t q0, int64_t q1,
                           const int64_t* __restrict__ pre, const int64_t* __restrict__ preu,
                           char* ubase, char* vbase, int esz, uint64_t* __restrict__ Uptr,
                           uint64_t* __restrict__ Vptr)
{
    int64_t q = q0 + (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= q1) return;
    uint32_t b = order[q];
    const int64_t u0 = preu[q0], v0 = pre[q0] - preu[q0];
    Uptr[b] = (uint64_t)(ubase + (preu[q] - u0) * esz);
    Vptr[b] = (uint64_t)(vbase + (pre[q] - preu[q] - v0) * esz);
}

__global__ void k_final_size(const Blk* __restrict__ blk, const uint32_t* __restrict__ order,
                             int64_t q0, int64_t q1, const int32_t* __restrict__ rank,
                             int64_t* __restrict__ fsu, int64_t* __restrict__ fsv)
{
    int64_t q = q0 + (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q >= q1) return;
    uint32_t b = order[q];
    fsu[q - q0] = (int64_t)rank[b] * blk[b].m;
    fsv[q - q0] = (int64_t)rank[b] * blk[b].n;
}

// Copy the rank-k columns of U and V (contiguous prefixes of the column-major
// scratch) into exactly sized U and V segments; one CTA per block.
__global__ void k_copy_factors(const Blk* __restrict__ blk, const uint32_t* __restrict__ order,
                               int64_t q0, int64_t q1, const int32_t* __restrict__ rank,
                               const int64_t* __restrict__ foffu, const int64_t* __restrict__ foffv,
                               char* ubase, char* vbase, int esz, uint64_t* __restrict__ Uptr,
                               uint64_t* __restrict__ Vptr)
{
    const int64_t w = blockIdx.x;
    const int lane = threadIdx.x;
    const int64_t q = q0 + w;
    if (q >= q1) return;
    uint32_t b = order[q];
    const Blk B = blk[b];
    const int r = rank[b];
    char* du = ubase + foffu[w] * esz;
    char* dv = vbase + foffv[w] * esz;
    const int64_t nu = (int64_t)r * B.m, nv = (int64_t)r * B.n;
    if (esz == 8) {
        const double* a = reinterpret_cast<const double*>(Uptr[b]);
        const double* c = reinterpret_cast<const double*>(Vptr[b]);
        for (int64_t e = lane; e < nu; e += NT) reinterpret_cast<double*>(du)[e] = a[e];
        for (int64_t e = lane; e < nv; e += NT) reinterpret_cast<double*>(dv)[e] = c[e];
    } else {
        const float* a = reinterpret_cast<const float*>(Uptr[b]);
        const float* c = reinterpret_cast<const float*>(Vptr[b]);
        for (int64_t e = lane; e < nu; e += NT) reinterpret_cast<float*>(du)[e] = a[e];
        for (int64_t e = lane; e < nv; e += NT) reinterpret_cast<float*>(dv)[e] = c[e];
    }
    __syncthreads();
    if (lane == 0) {
        Uptr[b] = (uint64_t)du;
        Vptr[b] = (uint64_t)dv;
    }
}


// Statistics of the factors: [sum rank, max rank, cap hits, mispredicted,
// rejected, factor entries, reserved entries, sum k m, evaluations,
// sum 2 k (k-1) (m + n)]
constexpr int NSTAT = 11;
__global__ void k_rank_stats(const Blk* __restrict__ blk, const int32_t* __restrict__ rank,
                             const int32_t* __restrict__ nrej, const int32_t* __restrict__ flags,
                             const int32_t* __restrict__ kres, int64_t n,
                             unsigned long long* __restrict__ out)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    unsigned long long s[NSTAT] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (b < n) {
        const unsigned long long r = rank[b], m = blk[b].m, nn = blk[b].n;
        const bool own = !(flags[b] & MIRROR_FLAG);   // compressed by its own ACA
        s[0] = r;
        s[1] = r;
        s[2] = own && (flags[b] & 2) ? 1 : 0;
        s[3] = own && (flags[b] & 1) ? 1 : 0;
        s[4] = own ? nrej[b] : 0;
        s[5] = r * (m + nn);
        s[6] = own ? (unsigned long long)kres[b] * (m + nn) : 0ull;
        s[7] = r * m;
        s[8] = own ? r * (m + nn) + (unsigned long long)nrej[b] * m : 0ull;
        s[9] = own && r ? 2ull * r * (r - 1) * (m + nn) : 0ull;
        s[10] = blk[b].row0 < blk[b].col0 ? r * nn : 0ull;   // V of the canonical blocks
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < NSTAT; ++k) {
            unsigned long long v = __shfl_xor_sync(0xffffffffu, s[k], o);
            s[k] = (k == 1) ? max(s[k], v) : s[k] + v;
        }
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < NSTAT; ++k)
            if (k == 1) atomicMax(&out[1], s[1]);
            else atomicAdd(&out[k], s[k]);
    }
}

struct Timer {
    cudaEvent_t a, b;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st)
    {
        HM_CUDA(cudaEventCreate(&a));
        HM_CUDA(cudaEventCreate(&b));
        HM_CUDA(cudaEventRecord(a, s));
    }
    double stop_ms()
    {
        HM_CUDA(cudaEventRecord(b, s));
        HM_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        HM_CUDA(cudaEventElapsedTime(&ms, a, b));
        return ms;
    }
    ~Timer()
    {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// Side streams for the ACA size classes, forked from and joined into s, with
// a pair of timing events per class.
struct ClassStreams {
    cudaStream_t main;
    cudaStream_t st[ACA_NCLASS];
    cudaEvent_t ev[ACA_NCLASS + 1];
    cudaEvent_t t0[ACA_NCLASS], t1[ACA_NCLASS];
    bool timed[ACA_NCLASS] = {};
    explicit ClassStreams(cudaStream_t s) : main(s)
    {
        for (int c = 0; c < ACA_NCLASS; ++c) {
            HM_CUDA(cudaStreamCreateWithFlags(&st[c], cudaStreamNonBlocking));
            HM_CUDA(cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming));
            HM_CUDA(cudaEventCreate(&t0[c]));
            HM_CUDA(cudaEventCreate(&t1[c]));
        }
        HM_CUDA(cudaEventCreateWithFlags(&ev[ACA_NCLASS], cudaEventDisableTiming));
    }
    // add the recorded class times to ms[] (synchronises the events)
    void collect(double* ms)
    {
        for (int c = 0; c < ACA_NCLASS; ++c) {
            if (!timed[c]) continue;
            HM_CUDA(cudaEventSynchronize(t1[c]));
            float x = 0.f;
            HM_CUDA(cudaEventElapsedTime(&x, t0[c], t1[c]));
            ms[c] += x;
            timed[c] = false;
        }
    }
    void fork()
    {
        HM_CUDA(cudaEventRecord(ev[ACA_NCLASS], main));
        for (int c = 0; c < ACA_NCLASS; ++c) HM_CUDA(cudaStreamWaitEvent(st[c], ev[ACA_NCLASS], 0));
    }
    void join()
    {
        for (int c = 0; c < ACA_NCLASS; ++c) {
            HM_CUDA(cudaEventRecord(ev[c], st[c]));
            HM_CUDA(cudaStreamWaitEvent(main, ev[c], 0));
        }
    }
    ~ClassStreams()
    {
        for (int c = 0; c < ACA_NCLASS; ++c) {
            cudaStreamSynchronize(st[c]);
            cudaStreamDestroy(st[c]);
            cudaEventDestroy(ev[c]);
            cudaEventDestroy(t0[c]);
            cudaEventDestroy(t1[c]);
        }
        cudaEventDestroy(ev[ACA_NCLASS]);
    }
};

void check_status(hm_handle_s& h)
{
    int st = 0;
    HM_CUDA(cudaMemcpyAsync(&st, h.status.p, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    HM_CUDA(cudaStreamSynchronize(h.stream));
    if (st) fail(HM_ETIMEOUT, "a device loop reached its iteration limit");
}

}  // namespace

void alloc_factor_meta(hm_handle_s& h)
{
    cudaStream_t s = h.stream;
    const int64_t n = std::max<int64_t>(h.n_adm, 1);
    h.kres.alloc(n, s);
    h.rank.alloc(n, s);
    h.nrej.alloc(n, s);
    h.flags.alloc(n, s);
    h.Uptr.alloc(n, s);
    h.Vptr.alloc(n, s);
    HM_CUDA(cudaMemsetAsync(h.flags.p, 0, n * sizeof(int32_t), s));
    HM_CUDA(cudaMemsetAsync(h.rank.p, 0, n * sizeof(int32_t), s));
    HM_CUDA(cudaMemsetAsync(h.nrej.p, 0, n * sizeof(int32_t), s));
}

// ACA of the admissible blocks ids[0..n) (all blocks when ids is null); see
// the file comment for the two storage modes (kpred != null: learned sizing,
// one arena; else bounded scratch passes with exact final segments).
// Blocks ids[0..n) in size-class order (the largest class first) with their
// reservations: kres (m + n) entries in all, kres m of them for U.
struct AcaOrder {
    int64_t n = 0;
    DevBuf<uint32_t> order;
    DevBuf<int64_t> pre, preu;
    std::vector<int64_t> hpre, hpreu;   // host copies of pre / preu (when asked for)
    int64_t tot = 0, totu = 0;           // pre[n], preu[n]
    int64_t cstart[ACA_NCLASS][ACA_NKB], cend[ACA_NCLASS][ACA_NKB];
};

// host_prefix: copy the whole reservation prefixes to the host (the bounded
// scratch passes and batch limits cut ranges by them); else only the totals.
void aca_order(hm_handle_s& h, const uint32_t* ids, int64_t n, const int32_t* kpred, AcaOrder& O,
               bool host_prefix = true)
{
    cudaStream_t s = h.stream;
    O.n = n;
    DevBuf<uint64_t> key(n, s);
    O.order.alloc(n, s);
    DevBuf<int64_t> ccount(ACA_NCLASS * ACA_NKB, s);
    HM_CUDA(cudaMemsetAsync(ccount.p, 0, ACA_NCLASS * ACA_NKB * sizeof(int64_t), s));
    k_classes<<<grid_for(n), NT, 0, s>>>(h.ablk.p, ids, n, h.opt.k_cap, kpred, key.p, O.order.p,
                                         h.kres.p, ccount.p); note_launch();
    HM_LAUNCH("classes");
    radix_sort_u64_u32(key.p, O.order.p, n, bits_for(ACA_NCLASS * ACA_NKB), s);
    int64_t cc[ACA_NCLASS * ACA_NKB];
    HM_CUDA(cudaMemcpyAsync(cc, ccount.p, sizeof(cc), cudaMemcpyDeviceToHost, s));
    DevBuf<int64_t> res(n, s), resu(n, s);
    O.pre.alloc(n + 1, s);
    O.preu.alloc(n + 1, s);
    k_reserve<<<grid_for(n), NT, 0, s>>>(h.ablk.p, O.order.p, n, h.kres.p, res.p, resu.p); note_launch();
    scan_exclusive_i64(res.p, O.pre.p, n, O.pre.p + n, s);
    scan_exclusive_i64(resu.p, O.preu.p, n, O.preu.p + n, s);
    if (host_prefix) {
        O.hpre.resize(n + 1);
        O.hpreu.resize(n + 1);
        HM_CUDA(cudaMemcpyAsync(O.hpre.data(), O.pre.p, (n + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(O.hpreu.data(), O.preu.p, (n + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
    }
    int64_t t2[2] = {0, 0};
    HM_CUDA(cudaMemcpyAsync(&t2[0], O.pre.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaMemcpyAsync(&t2[1], O.preu.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    O.tot = t2[0];
    O.totu = t2[1];
    int64_t q = 0;
    for (int c = ACA_NCLASS - 1; c >= 0; --c)
        for (int kb = 0; kb < ACA_NKB; ++kb) {
            O.cstart[c][kb] = q;
            q += cc[c * ACA_NKB + kb];
            O.cend[c][kb] = q;
        }
}

// Arguments of the ACA kernels for this handle (setn keeps the per-set point
// counts of the mixed stopping floor alive).
AcaArgs aca_args(hm_handle_s& h, DevBuf<int64_t>& setn)
{
    cudaStream_t s = h.stream;
    AcaArgs a;
    a.blk = h.ablk.p;
    a.kres = h.kres.p;
    a.Uptr = h.Uptr.p;
    a.Vptr = h.Vptr.p;
    a.rank = h.rank.p;
    a.nrej = h.nrej.p;
    a.flags = h.flags.p;
    a.status = h.status.p;
    a.eps = h.aca_eps;
    a.aca_eta = h.opt.aca_eta;
    a.eps0 = h.opt.eps0 > 0 ? h.opt.eps0 : (h.precision == HM_PREC_FP64 ? 1e-14 : 1e-6);
    a.k_cap = h.opt.k_cap;
    a.bset = nullptr;
    a.step_limit = aca_step_limit();
    a.set_n = nullptr;
    // The mixed-precision floor m n / N rests on ||A||_F^2 >= N phi(0)^2 (the
    // diagonal of A_{phi, Y x Y}), so the floors of all blocks add up to at
    // most ||A||_F^2. Two sets have no diagonal; there F^2 = the dense leaves'
    // sum of squares, also a lower bound of ||A||_F^2, takes its place with
    // N1 N2 entries: floor m n F^2 / (N1 N2), i.e. N replaced by
    // ceil(N1 N2 / F^2). Without dense leaves (F^2 = 0) no floor is used.
    const bool floor = h.precision == HM_PREC_MIXED && (!h.rect || h.rect_fro2 > 0.0);
    if (floor) {
        std::vector<int64_t> sn(h.sets.size());
        for (size_t q = 0; q < h.sets.size(); ++q) sn[q] = h.sets[q].N;
        if (h.rect)
            sn[0] = std::max<int64_t>(
                1, (int64_t)std::ceil((double)h.n_rows * (double)h.n_cols / h.rect_fro2));
        setn.alloc(sn.size(), s);
        copy_in(setn.p, sn.data(), sn.size() * sizeof(int64_t), s);
        a.bset = h.adm_set.p;
        a.set_n = setn.p;
    }
    return a;
}

// ACA of the blocks O.order[q0..q1): every size class on its own stream so
// that the few largest blocks (clusters of CTAs) overlap the many small ones;
// profile = 2 runs the classes one after another on the main stream, so that
// each class's time is its kernels' own duration.
void aca_range(hm_handle_s& h, const AcaOrder& O, const AcaArgs& a, int64_t q0, int64_t q1)
{
    cudaStream_t s = h.stream;
    ClassStreams cs(s);
    const bool serial = h.opt.profile == 2;
    cs.fork();
    for (int c = ACA_NCLASS - 1; c >= 0; --c) {
        cudaStream_t sc = serial ? s : cs.st[c];
        bool any = false;
        for (int kb = 0; kb < ACA_NKB; ++kb) {
            int64_t lo = std::max(q0, O.cstart[c][kb]), hi = std::min(q1, O.cend[c][kb]);
            if (hi <= lo) continue;
            if (!any) HM_CUDA(cudaEventRecord(cs.t0[c], sc));
            any = true;
            const int64_t bs = aca_batch_entries();
            if (bs <= 0) {
                aca_run(h.precision, h.kp, h.X, a, O.order.p + lo, hi - lo, c, kb, h.max_set_n, sc);
                continue;
            }
            // batches of consecutive blocks with at most bs reserved entries
            for (int64_t b0 = lo; b0 < hi;) {
                int64_t b1 = std::upper_bound(O.hpre.begin() + b0 + 1, O.hpre.begin() + hi + 1,
                                              O.hpre[b0] + bs) - O.hpre.begin() - 1;
                b1 = std::max(b1, b0 + 1);
                aca_run(h.precision, h.kp, h.X, a, O.order.p + b0, b1 - b0, c, kb, h.max_set_n, sc);
                b0 = b1;
            }
        }
        if (any) {
            HM_CUDA(cudaEventRecord(cs.t1[c], sc));
            cs.timed[c] = true;
        }
    }
    cs.join();
    cs.collect(h.stats.t_aca_class_ms);
}

// Entries of the automatic ACA scratch: 30 % of the free device memory.
int64_t scratch_entries(hm_handle_s& h, int esz)
{
    size_t freeb = 0, totb = 0;
    HM_CUDA(cudaMemGetInfo(&freeb, &totb));
    const int64_t cap = h.opt.scratch_gb > 0 ? (int64_t)(h.opt.scratch_gb * 1e9 / esz)
                                             : (int64_t)(0.30 * (double)freeb / esz);
    return std::max<int64_t>(cap, 1);
}

// ACA of the admissible blocks ids[0..n) (all blocks when ids is null); see
// the file comment for the two storage modes (kpred != null: learned sizing,
// one arena; else bounded scratch passes with exact final segments).
// keep_reserved: when one scratch pass holds every block, the scratch itself
// becomes the blocks' storage (their rank-k columns are the prefixes of their
// reservations), with no copy into exact segments; used for the few blocks a
// rank model under-predicted.
void compress(hm_handle_s& h, const uint32_t* ids, int64_t n, const int32_t* kpred,
              bool keep_reserved)
{
    cudaStream_t s = h.stream;
    const int esz = h.precision == HM_PREC_FP64 ? 8 : 4;
    if (n == 0) return;
    AcaOrder O;
    // learned sizing needs only the totals on the host, unless batch limits
    // cut the class ranges by the prefixes
    aca_order(h, ids, n, kpred, O, !kpred || aca_batch_entries() > 0);
    const std::vector<int64_t>& hpre = O.hpre;
    const std::vector<int64_t>& hpreu = O.hpreu;
    DevBuf<int64_t> setn;
    const AcaArgs a = aca_args(h, setn);

    if (kpred) {
        // learned sizing: reserve the predicted ranks directly (no copy)
        auto useg = std::make_unique<FactorSegment>();
        auto vseg = std::make_unique<FactorSegment>();
        useg->mem.alloc((size_t)std::max<int64_t>(O.totu, 1) * esz, s);
        vseg->mem.alloc((size_t)std::max<int64_t>(O.tot - O.totu, 1) * esz, s);
        k_set_ptrs<<<grid_for(n), NT, 0, s>>>(O.order.p, 0, n, O.pre.p, O.preu.p, useg->mem.p,
                                               vseg->mem.p, esz, h.Uptr.p, h.Vptr.p); note_launch();
        HM_LAUNCH("set ptrs");
        h.usegments.push_back(std::move(useg));
        h.vsegments.push_back(std::move(vseg));
        aca_range(h, O, a, 0, n);
        h.stats.aca_passes += 1;
        return;
    }

    int64_t cap = scratch_entries(h, esz);
    int64_t maxres = 0;
    for (int64_t q = 0; q < n; ++q) maxres = std::max(maxres, hpre[q + 1] - hpre[q]);
    cap = std::max(cap, maxres);
    cap = std::min(cap, hpre[n]);
    DevBuf<char> scratch((size_t)cap * esz, s);
    int passes = 0;
    for (int64_t q0 = 0; q0 < n;) {
        // largest q1 with hpre[q1] - hpre[q0] <= cap
        int64_t q1 = std::upper_bound(hpre.begin() + q0 + 1, hpre.end(), hpre[q0] + cap) -
                     hpre.begin() - 1;
        q1 = std::max(q1, q0 + 1);
        // the chunk's U reservations first, then its V reservations
        char* vbase = scratch.p + (hpreu[q1] - hpreu[q0]) * esz;
        k_set_ptrs<<<grid_for(q1 - q0), NT, 0, s>>>(O.order.p, q0, q1, O.pre.p, O.preu.p,
                                                     scratch.p, vbase, esz, h.Uptr.p, h.Vptr.p); note_launch();
        HM_LAUNCH("set ptrs");
        aca_range(h, O, a, q0, q1);
        if (keep_reserved && q0 == 0 && q1 == n) {
            // kept in the V segments, which live as long as the handle
            auto seg = std::make_unique<FactorSegment>();
            seg->mem = std::move(scratch);
            h.vsegments.push_back(std::move(seg));
            ++passes;
            break;
        }
        const int64_t nq = q1 - q0;
        DevBuf<int64_t> fsu(nq, s), fsv(nq, s), foffu(nq + 1, s), foffv(nq + 1, s);
        k_final_size<<<grid_for(nq), NT, 0, s>>>(h.ablk.p, O.order.p, q0, q1, h.rank.p, fsu.p, fsv.p); note_launch();
        scan_exclusive_i64(fsu.p, foffu.p, nq, foffu.p + nq, s);
        scan_exclusive_i64(fsv.p, foffv.p, nq, foffv.p + nq, s);
        int64_t tot[2] = {0, 0};
        HM_CUDA(cudaMemcpyAsync(&tot[0], foffu.p + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(&tot[1], foffv.p + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        auto useg = std::make_unique<FactorSegment>();
        auto vseg = std::make_unique<FactorSegment>();
        useg->mem.alloc((size_t)std::max<int64_t>(tot[0], 1) * esz, s);
        vseg->mem.alloc((size_t)std::max<int64_t>(tot[1], 1) * esz, s);
        k_copy_factors<<<(unsigned)nq, NT, 0, s>>>(h.ablk.p, O.order.p, q0, q1, h.rank.p, foffu.p,
                                                   foffv.p, useg->mem.p, vseg->mem.p, esz,
                                                   h.Uptr.p, h.Vptr.p); note_launch();
        HM_LAUNCH("copy factors");
        h.usegments.push_back(std::move(useg));
        h.vsegments.push_back(std::move(vseg));
        ++passes;
        q0 = q1;
    }
    h.stats.aca_passes += passes;
}

__global__ void k_iota_u32(uint32_t* __restrict__ ids, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q < n) ids[q] = (uint32_t)q;
}

__global__ void k_full_reserve(const Blk* __restrict__ blk, int64_t n, int kcap,
                               int64_t* __restrict__ res)
{
    const int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    const Blk B = blk[b];
    res[b] = (int64_t)min(kcap, min(B.m, B.n)) * (B.m + B.n);
}

__global__ void k_pred_reserve(const Blk* __restrict__ blk, int64_t n, int kcap,
                               const int32_t* __restrict__ kpred, int64_t* __restrict__ res)
{
    const int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    const Blk B = blk[b];
    res[b] = (int64_t)aca_reservation(B.m, B.n, kcap, kpred, b) * (B.m + B.n);
}

// Blocks of ids[0..n) whose reservation was too small (flag bit 0).
__global__ void k_np_mispred(const uint32_t* __restrict__ ids, int64_t n,
                             const int32_t* __restrict__ flags, int64_t* __restrict__ f)
{
    const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q < n) f[q] = (flags[ids[q]] & 1) ? 1 : 0;
}

__global__ void k_np_mispred_ids(const uint32_t* __restrict__ ids, int64_t n,
                                 const int64_t* __restrict__ f, const int64_t* __restrict__ off,
                                 uint32_t* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (q < n && f[q]) out[off[q]] = ids[q];
}

// On-the-fly mode, at build time: passes of consecutive admissible leaves
// (block order) whose full reservations min(k_cap, m, n) (m + n) fit the
// scratch bound, and the buffers every product reuses.
void np_prepare(hm_handle_s& h)
{
    cudaStream_t s = h.stream;
    const int64_t n = h.n_adm;
    const int esz = h.precision == HM_PREC_FP64 ? 8 : 4;
    h.np_pass.assign(1, 0);
    h.np_ids.alloc(std::max<int64_t>(n, 1), s);
    int64_t cap = 1, most = 1;
    std::vector<int64_t> partner;   // symmetric: canonical partner of every leaf
    if (n > 0) {
        k_iota_u32<<<grid_for(n), NT, 0, s>>>(h.np_ids.p, n); note_launch();
        DevBuf<int64_t> res(n, s);
        if (h.opt.rank_model) {
            // the learned model sizes every leaf's reservation (the passes
            // then hold more leaves); a block whose prediction is too small
            // is re-run inside its pass with the full reservation
            h.np_kpred.alloc(n, s);
            predict_ranks(h, h.np_kpred.p);
            k_pred_reserve<<<grid_for(n), NT, 0, s>>>(h.ablk.p, n, h.opt.k_cap, h.np_kpred.p,
                                                      res.p); note_launch();
        } else {
            k_full_reserve<<<grid_for(n), NT, 0, s>>>(h.ablk.p, n, h.opt.k_cap, res.p); note_launch();
        }
        HM_LAUNCH("np reservations");
        std::vector<int64_t> hr(n);
        HM_CUDA(cudaMemcpyAsync(hr.data(), res.p, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        if (h.opt.symmetric) {
            // mirror leaves reserve nothing: they take their partner's factors
            DevBuf<int64_t> dp(n, s);
            k_np_partner<<<grid_for(n), NT, 0, s>>>(h.ablk.p, n, dp.p, h.status.p); note_launch();
            HM_LAUNCH("np partners");
            partner.resize(n);
            HM_CUDA(cudaMemcpyAsync(partner.data(), dp.p, n * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            check_status(h);
            for (int64_t b = 0; b < n; ++b)
                if (partner[b] != b) hr[b] = 0;
        }
        int64_t total = 0, maxres = 0;
        for (int64_t b = 0; b < n; ++b) {
            total += hr[b];
            maxres = std::max(maxres, hr[b]);
        }
        cap = std::min(std::max(scratch_entries(h, esz), maxres), std::max<int64_t>(total, 1));
        int64_t acc = 0, first = 0;
        for (int64_t b = 0; b < n; ++b) {
            if (acc + hr[b] > cap && b > first) {
                h.np_pass.push_back(b);
                most = std::max(most, b - first);
                first = b;
                acc = 0;
            }
            acc += hr[b];
        }
        h.np_pass.push_back(n);
        most = std::max(most, n - first);
    }
    h.np_kcap = std::max(h.opt.k_cap, 1);
    h.np_scratch.alloc((size_t)cap * esz, s);
    h.np_xm.alloc((size_t)std::max<int64_t>(h.Ntot, 1) * esz, s);
    h.np_yacc.alloc(std::max<int64_t>(h.Ntot, 1), s);
    h.np_ld = std::max(h.leaf, 1);
    h.np_part.alloc((size_t)std::max<int64_t>(h.lists.n_items, 1) * h.np_ld, s);
    np_lists(h.ablk.p, n, h.lists.lr_ptr.p, h.n_tiles, h.np_vptr, h.np_vitems, h.np_aptr,
             h.np_aitems, h.np_hvptr, h.np_naitems, s);
    int64_t most_items = 1;
    if (h.opt.symmetric && n > 0) {
        // pass q: the canonical leaves of its block range and their mirrors
        const int64_t P = (int64_t)h.np_pass.size() - 1;
        std::vector<int32_t> pid(n), tix(n);
        for (int64_t q = 0; q < P; ++q)
            for (int64_t b = h.np_pass[q]; b < h.np_pass[q + 1]; ++b)
                if (partner[b] == b) pid[b] = (int32_t)q;
        std::vector<uint32_t> cids;
        h.np_cptr.assign(P + 1, 0);
        for (int64_t q = 0; q < P; ++q) {
            h.np_cptr[q] = (int64_t)cids.size();
            for (int64_t b = h.np_pass[q]; b < h.np_pass[q + 1]; ++b)
                if (partner[b] == b) cids.push_back((uint32_t)b);
        }
        h.np_cptr[P] = (int64_t)cids.size();
        for (int64_t b = 0; b < n; ++b)
            if (partner[b] != b) pid[b] = pid[partner[b]];
        h.np_pbptr.assign(P + 1, 0);
        for (int64_t b = 0; b < n; ++b) ++h.np_pbptr[pid[b] + 1];
        for (int64_t q = 0; q < P; ++q) h.np_pbptr[q + 1] += h.np_pbptr[q];
        std::vector<int64_t> pblk(n), fill(h.np_pbptr.begin(), h.np_pbptr.end() - 1);
        for (int64_t b = 0; b < n; ++b) {
            const int64_t at = fill[pid[b]]++;
            pblk[at] = b;
            tix[b] = (int32_t)(at - h.np_pbptr[pid[b]]);
        }
        std::vector<int64_t> pitems, pfirst(n, 0);
        pitems.reserve(h.np_hvptr[n]);
        h.np_piptr.assign(P + 1, 0);
        most = 1;
        for (int64_t q = 0; q < P; ++q) {
            h.np_piptr[q] = (int64_t)pitems.size();
            for (int64_t at = h.np_pbptr[q]; at < h.np_pbptr[q + 1]; ++at) {
                const int64_t b = pblk[at];
                pfirst[b] = (int64_t)pitems.size() - h.np_piptr[q];
                for (int64_t it = h.np_hvptr[b]; it < h.np_hvptr[b + 1]; ++it) pitems.push_back(it);
            }
            most = std::max(most, h.np_pbptr[q + 1] - h.np_pbptr[q]);
            most_items = std::max(most_items, (int64_t)pitems.size() - h.np_piptr[q]);
        }
        h.np_piptr[P] = (int64_t)pitems.size();
        copy_in(h.np_ids.p, cids.data(), cids.size() * sizeof(uint32_t), s);
        h.np_passid.alloc(n, s);
        h.np_tidx.alloc(n, s);
        h.np_pblk.alloc(n, s);
        h.np_pfirst.alloc(n, s);
        h.np_pitems.alloc(std::max<size_t>(pitems.size(), 1), s);
        copy_in(h.np_passid.p, pid.data(), n * sizeof(int32_t), s);
        copy_in(h.np_tidx.p, tix.data(), n * sizeof(int32_t), s);
        copy_in(h.np_pblk.p, pblk.data(), n * sizeof(int64_t), s);
        copy_in(h.np_pfirst.p, pfirst.data(), n * sizeof(int64_t), s);
        copy_in(h.np_pitems.p, pitems.data(), pitems.size() * sizeof(int64_t), s);
        HM_CUDA(cudaStreamSynchronize(s));
    } else {
        for (size_t q = 0; q + 1 < h.np_pass.size(); ++q)
            most_items = std::max(most_items, h.np_hvptr[h.np_pass[q + 1]] - h.np_hvptr[h.np_pass[q]]);
    }
    h.np_t.alloc((size_t)most * h.np_kcap * esz, s);
    h.np_tp.alloc((size_t)most_items * h.np_kcap * esz, s);
    h.np_acc.alloc((size_t)std::max<int64_t>(h.np_naitems, 1) * h.np_ld, s);
    HM_CUDA(cudaStreamSynchronize(s));
}

namespace {
void rank_stats(hm_handle_s& h);
}

// y = H x (+ sigma^2 x) for device x, y without stored factors: per pass, ACA
// of its leaves into the scratch, then t_b = V_b^T x|sigma and y_m += U_b t_b;
// then the dense leaves evaluated on the fly. Runs on the handle's stream,
// ordered after and before stream s.
// Rank model in the on-the-fly mode: the blocks of one pass (ids[0..n)) whose
// predicted reservation was too small run again with the full one, in memory
// of their own that lives until the product ends.
void np_rerun(hm_handle_s& h, const uint32_t* ids, int64_t n, const AcaArgs& a, int esz,
              std::vector<DevBuf<char>>& keep)
{
    cudaStream_t s = h.stream;
    DevBuf<int64_t> f(n, s), off(n + 1, s);
    k_np_mispred<<<grid_for(n), NT, 0, s>>>(ids, n, h.flags.p, f.p); note_launch();
    scan_exclusive_i64(f.p, off.p, n, off.p + n, s);
    int64_t cnt = 0;
    HM_CUDA(cudaMemcpyAsync(&cnt, off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    if (cnt == 0) return;
    h.np_mispredicted += cnt;
    DevBuf<uint32_t> mis(cnt, s);
    k_np_mispred_ids<<<grid_for(n), NT, 0, s>>>(ids, n, f.p, off.p, mis.p); note_launch();
    HM_LAUNCH("np mispredicted ids");
    AcaOrder O;
    aca_order(h, mis.p, cnt, nullptr, O, aca_batch_entries() > 0);
    DevBuf<char> mem((size_t)std::max<int64_t>(O.tot, 1) * esz, s);
    char* vbase = mem.p + O.totu * esz;
    k_set_ptrs<<<grid_for(cnt), NT, 0, s>>>(O.order.p, 0, cnt, O.pre.p, O.preu.p, mem.p, vbase,
                                            esz, h.Uptr.p, h.Vptr.p); note_launch();
    HM_LAUNCH("set ptrs");
    aca_range(h, O, a, 0, cnt);
    keep.push_back(std::move(mem));
}

void np_matvec(hm_handle_s& h, const double* x, double* y, int accumulate, cudaStream_t s)
{
    cudaStream_t hs = h.stream;
    cudaEvent_t ev = nullptr;
    if (s != hs) {
        HM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        HM_CUDA(cudaEventRecord(ev, s));
        HM_CUDA(cudaStreamWaitEvent(hs, ev, 0));
    }
    const int64_t N = h.Ntot;
    const int esz = h.precision == HM_PREC_FP64 ? 8 : 4;
    HM_CUDA(cudaMemsetAsync(h.np_yacc.p, 0, N * sizeof(double), hs));
    HM_CUDA(cudaMemsetAsync(h.np_acc.p, 0, h.np_acc.bytes(), hs));
    np_gather_x(h.precision, x, h.perm.p, N, h.np_xm.p, hs);
    DevBuf<int64_t> setn;
    const AcaArgs a = aca_args(h, setn);
    // profile = 1: events on the handle's stream around every phase (ACA and
    // low-rank apply of each pass, then the dense leaves)
    const bool prof = h.opt.profile != 0;
    const size_t npass = h.np_pass.size() - 1;
    std::vector<cudaEvent_t> pe;
    auto mark = [&]() {
        if (!prof) return;
        cudaEvent_t e;
        HM_CUDA(cudaEventCreate(&e));
        HM_CUDA(cudaEventRecord(e, hs));
        pe.push_back(e);
    };
    mark();
    const bool sym = h.opt.symmetric;
    std::vector<DevBuf<char>> rerun_mem;   // factors of re-run blocks, kept to the end
    for (size_t q = 0; q < npass; ++q) {
        // the leaves compressed in this pass: its block range, or only the
        // canonical ones of it (symmetric)
        const int64_t c0 = sym ? h.np_cptr[q] : h.np_pass[q];
        const int64_t nb = (sym ? h.np_cptr[q + 1] : h.np_pass[q + 1]) - c0;
        if (nb > 0) {
            const int32_t* kp = h.opt.rank_model ? h.np_kpred.p : nullptr;
            AcaOrder O;
            aca_order(h, h.np_ids.p + c0, nb, kp, O, aca_batch_entries() > 0);
            // the pass's reservations must fit the scratch they were cut for
            if (O.tot * esz > (int64_t)h.np_scratch.n)
                fail(HM_EOVERFLOW, "on-the-fly pass reserves more than its scratch");
            char* vbase = h.np_scratch.p + O.totu * esz;
            k_set_ptrs<<<grid_for(nb), NT, 0, hs>>>(O.order.p, 0, nb, O.pre.p, O.preu.p,
                                                     h.np_scratch.p, vbase, esz, h.Uptr.p, h.Vptr.p); note_launch();
            HM_LAUNCH("set ptrs");
            aca_range(h, O, a, 0, nb);
            if (kp) np_rerun(h, h.np_ids.p + c0, nb, a, esz, rerun_mem);
        }
        if (sym) {
            // mirror leaves take their partners' factors (those of this pass
            // are applied now; the others are reset in their partners' pass)
            k_mirror<<<grid_for(h.n_adm), NT, 0, hs>>>(h.ablk.p, h.n_adm, h.Uptr.p, h.Vptr.p,
                                                       h.rank.p, h.nrej.p, h.flags.p,
                                                       h.status.p); note_launch();
            HM_LAUNCH("np mirror leaves");
        }
        mark();
        if (sym) {
            NpSymPass sp;
            sp.pitems = h.np_pitems.p;
            sp.pblk = h.np_pblk.p;
            sp.pfirst = h.np_pfirst.p;
            sp.passid = h.np_passid.p;
            sp.tidx = h.np_tidx.p;
            sp.q = (int)q;
            np_lowrank(h.precision, h.ablk.p, h.rank.p, h.Uptr.p, h.Vptr.p, h.np_pbptr[q],
                       h.np_pbptr[q + 1], h.np_vptr.p, h.np_vitems.p, h.np_piptr[q],
                       h.np_piptr[q + 1], h.np_aitems.p, h.np_naitems, h.lists.lr_ent.p,
                       h.tile_m.p, h.np_xm.p, h.np_tp.p, h.np_t.p, h.np_kcap, h.np_ld,
                       h.np_acc.p, hs, &sp);
        } else {
            const int64_t b0 = h.np_pass[q], b1 = h.np_pass[q + 1];
            np_lowrank(h.precision, h.ablk.p, h.rank.p, h.Uptr.p, h.Vptr.p, b0, b1, h.np_vptr.p,
                       h.np_vitems.p, h.np_hvptr[b0], h.np_hvptr[b1], h.np_aitems.p,
                       h.np_naitems, h.lists.lr_ent.p, h.tile_m.p, h.np_xm.p, h.np_tp.p,
                       h.np_t.p, h.np_kcap, h.np_ld, h.np_acc.p, hs);
        }
        mark();
    }
    check_status(h);
    h.stats.n_mispredicted = h.np_mispredicted;
    np_apply_finish(h.np_aptr.p, h.tile_row0.p, h.tile_m.p, h.n_tiles, h.np_ld, h.np_acc.p,
                    h.np_yacc.p, hs);
    mark();
    np_near(h.precision, h.kp, h.X, h.lists.items.p, h.lists.n_items, h.lists.item_ptr.p,
            h.lists.ucol_ptr.p, h.lists.ncol_ptr.p, h.lists.ncol_x.p, h.tile_row0.p, h.tile_m.p,
            h.n_tiles, h.np_ld, h.np_xm.p, h.np_part.p, h.np_yacc.p, hs);
    mark();
    np_finish(h.perm.p, nullptr, h.sigma2, N, h.np_yacc.p, x, y, accumulate, hs);
    mark();
    if (prof) {
        // pe: start, then (after ACA, after low-rank) per pass, before and
        // after the dense leaves, end
        HM_CUDA(cudaEventSynchronize(pe.back()));
        auto ms = [&](size_t i, size_t j) {
            float t = 0.f;
            HM_CUDA(cudaEventElapsedTime(&t, pe[i], pe[j]));
            return (double)t;
        };
        for (size_t q = 0; q < npass; ++q) {
            h.stats.t_np_aca_ms += ms(q == 0 ? 0 : 2 * q, 2 * q + 1);
            h.stats.t_np_lowrank_ms += ms(2 * q + 1, 2 * q + 2);
        }
        const size_t k0 = 2 * npass + 1;
        h.stats.t_np_near_ms += ms(k0, k0 + 1);
        h.stats.t_mvp_ms += ms(0, pe.size() - 1);
        h.stats.mvp_count += 1;
        for (cudaEvent_t e : pe) cudaEventDestroy(e);
        rank_stats(h);      // the ACA work of this product (ranks, evaluations, flops)
    }
    if (ev) {
        HM_CUDA(cudaEventRecord(ev, hs));
        HM_CUDA(cudaStreamWaitEvent(s, ev, 0));
        cudaEventDestroy(ev);
    }
}

namespace {

void rank_stats(hm_handle_s& h)
{
    cudaStream_t s = h.stream;
    DevBuf<unsigned long long> out(NSTAT, s);
    HM_CUDA(cudaMemsetAsync(out.p, 0, NSTAT * sizeof(unsigned long long), s));
    if (h.n_adm > 0)
        k_rank_stats<<<grid_for(h.n_adm), NT, 0, s>>>(h.ablk.p, h.rank.p, h.nrej.p, h.flags.p,
                                                     h.kres.p, h.n_adm, out.p); note_launch();
    unsigned long long o[NSTAT];
    HM_CUDA(cudaMemcpyAsync(o, out.p, sizeof(o), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    h.stats.sum_rank = (int64_t)o[0];
    h.stats.max_rank = (int)o[1];
    h.stats.rank_cap_hits = (int64_t)o[2];
    h.stats.n_rejected = (int64_t)o[4];
    h.stats.factor_entries = (int64_t)o[5];
    h.stats.reserved_factor_entries = (int64_t)o[6];
    h.factor_entries_U = (int64_t)o[7];
    h.factor_entries_Vc = (int64_t)o[10];
    h.stats.aca_evals = (int64_t)o[8];
    // algorithmic flops of one kernel evaluation: squared distance in three
    // coordinates (3 subtractions, 1 multiply, 2 fused multiply-adds = 8)
    // plus the kernel (Gaussian: scale + exp = 2; Matern-3/2: sqrt, scale,
    // exp, add, multiply = 5; Matern K_1 within twice the length scale: its
    // two 13-term series (26 fused multiply-adds, 13 multiplies), log, add,
    // multiply = 68; farther entries take a quadrature of 12 to 20 terms)
    const double fe = h.kernel == HM_GAUSSIAN ? 10.0 : h.kernel == HM_MATERN32 ? 13.0 : 76.0;
    h.stats.aca_flops = fe * (double)o[8] + (double)o[9];
}

void validate(int nsets, const int64_t* N, const int* d, int kernel, const double* params,
              int leaf, double eta, const hm_options& o, bool rect)
{
    if (nsets < 1) fail(HM_EINVAL, "no point sets");
    if (!params) fail(HM_EINVAL, "params is NULL");
    if (kernel != HM_GAUSSIAN && kernel != HM_MATERN32 && kernel != HM_MATERN_K1)
        fail(HM_EINVAL, "unknown kernel");
    if (!(params[0] > 0.0) || !std::isfinite(params[0])) fail(HM_EINVAL, "length scale must be > 0");
    if (!(params[1] >= 0.0) || !std::isfinite(params[1])) fail(HM_EINVAL, "sigma^2 must be >= 0");
    if (leaf < 1) fail(HM_EINVAL, "leaf_size must be >= 1");
    if (!(eta >= 0.0) || !std::isfinite(eta)) fail(HM_EINVAL, "eta must be >= 0");
    if (o.k_cap < 1 || o.k_cap > 128) fail(HM_EINVAL, "k_cap must be in [1, 128]");
    if (o.precision != HM_PREC_FP64 && o.precision != HM_PREC_MIXED)
        fail(HM_EINVAL, "unknown precision");
    if (o.near_format < 0 || o.near_format > HM_NEAR_BF16) fail(HM_EINVAL, "unknown near format");
    if (o.precision == HM_PREC_FP64 && o.near_format != HM_NEAR_AUTO &&
        o.near_format != HM_NEAR_FP64)
        fail(HM_ENOTSUP, "the FP64 path stores the near field in FP64");
    if (o.symmetric < 0 || o.symmetric > 2) fail(HM_EINVAL, "symmetric must be 0, 1 or 2");
    int64_t tot = 0;
    for (int q = 0; q < nsets; ++q) {
        if (N[q] < 1) fail(HM_EINVAL, "N must be >= 1");
        if (d[q] < 1 || d[q] > 3) fail(HM_EINVAL, "d must be 1, 2 or 3");
        tot += N[q];
    }
    if (tot >= (1ll << 31)) fail(HM_EINVAL, "more than 2^31 points");
    if (o.row_hi > 0) {
        if (rect || nsets != 1)
            fail(HM_ENOTSUP, "a block-row share (row_lo, row_hi) is for one point set");
        if (o.row_lo < 0 || o.row_lo >= o.row_hi || o.row_hi > N[0])
            fail(HM_EINVAL, "row range must satisfy 0 <= row_lo < row_hi <= N");
    }
    if (o.on_the_fly && o.rank_model && rect)
        fail(HM_ENOTSUP, "the rank model needs one square point set");
    if (rect) {
        if (nsets != 2) fail(HM_EINVAL, "a rectangular matrix takes two point sets");
        if (d[0] != d[1]) fail(HM_EINVAL, "both point sets need the same dimension");
        if (params[1] != 0.0)
            fail(HM_EINVAL, "sigma^2 needs a square matrix (one set for rows and columns)");
        if (o.symmetric || o.rank_model)
            fail(HM_ENOTSUP, "symmetric mode and the rank model need a square matrix");
    }
}

}  // namespace

void build_sets(hm_handle_s& h, int nsets, const double* points_all, const int64_t* N,
                const int* d, int kernel, const double* params, int leaf, double eta,
                double aca_eps, const hm_options& opt, bool rect)
{
    validate(nsets, N, d, kernel, params, leaf, eta, opt, rect);
    if (!points_all) fail(HM_EINVAL, "points is NULL");
    auto t0 = std::chrono::steady_clock::now();
    h.opt = opt;
    h.kernel = kernel;
    h.ell = params[0];
    h.sigma2 = params[1];
    h.leaf = leaf;
    h.eta = eta;
    h.aca_eps = aca_eps;
    h.precision = opt.precision;
    h.near_format = opt.near_format == HM_NEAR_AUTO
                        ? (opt.precision == HM_PREC_FP64 ? HM_NEAR_FP64 : HM_NEAR_BF16X2)
                        : opt.near_format;
    // symmetric = 2: also store each off-diagonal dense leaf once (mixed
    // precision, a paired or FP32 near field, slices of at most 64 rows,
    // stored mode); otherwise it acts as symmetric = 1
    h.sym_near = opt.symmetric == 2 && opt.precision == HM_PREC_MIXED && !opt.on_the_fly &&
                 !rect && slice_ld(leaf) <= 64 && h.near_format != HM_NEAR_BF16 &&
                 h.near_format != HM_NEAR_FP64 ? 1 : 0;
    h.stream = (cudaStream_t)opt.stream;
    h.kp = make_kernel_params(kernel, h.ell);
    h.kp.dmax = 1;
    for (int q = 0; q < nsets; ++q) h.kp.dmax = std::max(h.kp.dmax, d[q]);
    cudaStream_t s = h.stream;
    h.status.alloc(1, s);
    HM_CUDA(cudaMemsetAsync(h.status.p, 0, sizeof(int), s));

    // sets, offsets, sizes
    int64_t Ntot = 0, nn = 0, nval = 0;
    h.sets.resize(nsets);
    for (int q = 0; q < nsets; ++q) {
        SetStructure& S = h.sets[q];
        S.N = N[q];
        S.d = d[q];
        S.C = leaf;
        S.depth = tree_depth(S.N, leaf);
        S.n_nodes = (2ll << S.depth) - 1;
        S.row0 = Ntot;
        S.node0 = nn;
        Ntot += S.N;
        nn += S.n_nodes;
        nval += S.N * S.d;
        h.max_set_n = std::max(h.max_set_n, S.N);
    }
    h.Ntot = Ntot;
    h.n_nodes_tot = nn;
    h.rect = rect;
    h.n_rows = rect ? N[0] : Ntot;
    h.n_cols = rect ? N[1] : Ntot;

    Timer tstruct(s);
    // points on the device
    DevBuf<double> pts_dev;
    const double* pts = points_all;
    if (!is_device_ptr(points_all)) {
        pts_dev.alloc(nval, s);
        copy_in(pts_dev.p, points_all, nval * sizeof(double), s);
        pts = pts_dev.p;
    }
    h.X64.alloc(3 * Ntot, s);
    h.X.x64[0] = h.X64.p;
    h.X.x64[1] = h.X64.p + Ntot;
    h.X.x64[2] = h.X64.p + 2 * Ntot;
    if (h.precision == HM_PREC_MIXED) {
        h.X32.alloc(6 * Ntot, s);
        h.X.x32 = h.X32.p;
        h.X.stride32 = Ntot;
    }
    h.perm.alloc(Ntot, s);
    h.codes.alloc(Ntot, s);
    h.node_lo.alloc(nn, s);
    h.node_hi.alloc(nn, s);
    h.bmin.alloc(3 * nn, s);
    h.bmax.alloc(3 * nn, s);

    std::vector<DevBuf<int2>> adm(nsets), dense(nsets);
    const double* p = pts;
    if (rect) {
        // both sets clustered on their own, Alg. 1 from (root of Y1, root of Y2)
        for (int q = 0; q < 2; ++q) {
            SetStructure& S = h.sets[q];
            build_tree(p, S, h.X, h.perm.p, h.codes.p + S.row0, h.node_lo.p, h.node_hi.p,
                       h.bmin.p, h.bmax.p, s);
            p += S.N * S.d;
        }
        traverse(h.sets[0], h.sets[1], eta, opt.adm_max, h.node_lo.p, h.node_hi.p, h.bmin.p,
                 h.bmax.p, adm[0], dense[0], s);
        h.sets[1].n_adm = h.sets[1].n_dense = 0;
        h.n_adm = h.sets[0].n_adm;
        h.n_dense = h.sets[0].n_dense;
    } else {
        for (int q = 0; q < nsets; ++q) {
            SetStructure& S = h.sets[q];
            build_structure(p, S, eta, opt.adm_max, h.X, h.perm.p, h.codes.p + S.row0,
                            h.node_lo.p, h.node_hi.p, h.bmin.p, h.bmax.p, adm[q], dense[q], s);
            p += S.N * S.d;
            if (opt.row_hi > 0) {
                // block-row share: the leaves whose rows meet [row_lo, row_hi)
                const int32_t* lo = h.node_lo.p + S.node0;
                const int32_t* hi = h.node_hi.p + S.node0;
                S.n_adm = row_filter(adm[q], S.n_adm, lo, hi, opt.row_lo, opt.row_hi,
                                     opt.symmetric, s);
                S.n_dense = row_filter(dense[q], S.n_dense, lo, hi, opt.row_lo, opt.row_hi,
                                       opt.symmetric, s);
            }
            h.n_adm += S.n_adm;
            h.n_dense += S.n_dense;
        }
    }
    for (const SetStructure& S : h.sets) h.stats.traversal_reruns += S.traversal_reruns;
    // perm holds set-local indices; make them absolute for the product
    // (the offsets are applied below by a small kernel per set)
    h.adm_pairs.alloc(std::max<int64_t>(h.n_adm, 1), s);
    h.dense_pairs.alloc(std::max<int64_t>(h.n_dense, 1), s);
    h.ablk.alloc(std::max<int64_t>(h.n_adm, 1), s);
    h.dblk.alloc(std::max<int64_t>(h.n_dense, 1), s);
    std::vector<DevBuf<int64_t>> trow(nsets);
    std::vector<DevBuf<int32_t>> tm(nsets);
    std::vector<int64_t> ntile(nsets);
    {
        int64_t ao = 0, dof = 0;
        for (int q = 0; q < nsets; ++q) {
            SetStructure& S = h.sets[q];
            const int32_t* lo = h.node_lo.p + S.node0;
            const int32_t* hi = h.node_hi.p + S.node0;
            // the column tree: set 1's for a rectangular matrix, else the same
            const SetStructure& Sc = rect ? h.sets[1] : S;
            const int32_t* lo2 = h.node_lo.p + Sc.node0;
            const int32_t* hi2 = h.node_hi.p + Sc.node0;
            if (S.n_adm) {
                HM_CUDA(cudaMemcpyAsync(h.adm_pairs.p + ao, adm[q].p, S.n_adm * sizeof(int2),
                                        cudaMemcpyDeviceToDevice, s));
                k_make_blk<<<grid_for(S.n_adm), NT, 0, s>>>(adm[q].p, S.n_adm, lo, hi, S.row0,
                                                            lo2, hi2, Sc.row0, h.ablk.p + ao); note_launch();
            }
            if (S.n_dense) {
                HM_CUDA(cudaMemcpyAsync(h.dense_pairs.p + dof, dense[q].p,
                                        S.n_dense * sizeof(int2), cudaMemcpyDeviceToDevice, s));
                k_make_blk<<<grid_for(S.n_dense), NT, 0, s>>>(dense[q].p, S.n_dense, lo, hi,
                                                              S.row0, lo2, hi2, Sc.row0,
                                                              h.dblk.p + dof); note_launch();
            }
            HM_LAUNCH("blocks");
            ao += S.n_adm;
            dof += S.n_dense;
            ntile[q] = 0;
            if (rect && q > 0) continue;   // the column set gives no rows
            // leaf tiles of this set, in row order
            DevBuf<int64_t> flag(S.n_nodes, s), off(S.n_nodes + 1, s);
            k_leaf_flags<<<grid_for(S.n_nodes), NT, 0, s>>>(lo, hi, S.n_nodes, leaf, flag.p); note_launch();
            scan_exclusive_i64(flag.p, off.p, S.n_nodes, off.p + S.n_nodes, s);
            int64_t nt = 0;
            HM_CUDA(cudaMemcpyAsync(&nt, off.p + S.n_nodes, sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            DevBuf<uint64_t> k(nt, s);
            DevBuf<uint32_t> v(nt, s);
            DevBuf<int32_t> vid(nt, s);
            k_leaf_emit<<<grid_for(S.n_nodes), NT, 0, s>>>(lo, hi, S.n_nodes, flag.p, off.p, k.p,
                                                           v.p, vid.p); note_launch();
            radix_sort_u64_u32(k.p, v.p, nt, bits_for(S.N + 1), s);
            trow[q].alloc(nt, s);
            tm[q].alloc(nt, s);
            k_leaf_tiles<<<grid_for(nt), NT, 0, s>>>(v.p, vid.p, nt, lo, hi, S.row0, trow[q].p,
                                                     tm[q].p); note_launch();
            HM_LAUNCH("tiles");
            ntile[q] = nt;
            h.n_tiles += nt;
        }
    }
    h.tile_row0.alloc(std::max<int64_t>(h.n_tiles, 1), s);
    h.tile_m.alloc(std::max<int64_t>(h.n_tiles, 1), s);
    {
        int64_t o = 0;
        for (int q = 0; q < nsets; ++q) {
            if (!ntile[q]) continue;
            HM_CUDA(cudaMemcpyAsync(h.tile_row0.p + o, trow[q].p, ntile[q] * sizeof(int64_t),
                                    cudaMemcpyDeviceToDevice, s));
            HM_CUDA(cudaMemcpyAsync(h.tile_m.p + o, tm[q].p, ntile[q] * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, s));
            o += ntile[q];
        }
    }
    fill_block_sets(h);
    add_perm_offsets(h);
    if (rect && h.precision == HM_PREC_MIXED)
        h.rect_fro2 = dense_fro2(h.kp, h.X, h.dblk.p, h.n_dense, s);
    h.stats.t_structure_ms = tstruct.stop_ms();
    adm.clear();
    dense.clear();
    if (pts_dev.p) pts_dev.release();

    if (opt.on_the_fly) {
        // no factors and no near field: the gather lists by tile and the
        // passes of the products
        alloc_factor_meta(h);
        mvp_build_lists(h.ablk.p, h.rank.p, h.n_adm, h.dblk.p, h.n_dense, h.tile_row0.p,
                        h.tile_m.p, h.n_tiles, h.lists, s);
        np_prepare(h);
        hm_stats& st = h.stats;
        st.n_points = Ntot;
        st.n_nodes = nn;
        st.n_adm = h.n_adm;
        st.n_dense = h.n_dense;
        st.n_tiles = h.n_tiles;
        st.depth = h.sets[0].depth;
        st.d = h.sets[0].d;
        st.precision = h.precision;
        st.near_format = h.near_format;
        st.aca_passes = (int)h.np_pass.size() - 1;
        st.near_entries = h.lists.near_elems;   // evaluated in every product
        st.t_total_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return;
    }
    if (opt.structure_only) {
        alloc_factor_meta(h);
        hm_stats& st = h.stats;
        st.n_points = Ntot;
        st.n_nodes = nn;
        st.n_adm = h.n_adm;
        st.n_dense = h.n_dense;
        st.n_tiles = h.n_tiles;
        st.depth = h.sets[0].depth;
        st.d = h.sets[0].d;
        st.precision = h.precision;
        st.near_format = h.near_format;
        HM_CUDA(cudaStreamSynchronize(s));
        return;
    }

    // batched ACA of the admissible leaves
    {
        Timer ta(s);
        alloc_factor_meta(h);
        DevBuf<int32_t> kpred;
        if (opt.rank_model) kpred.alloc(std::max<int64_t>(h.n_adm, 1), s);
        if (opt.rank_model && !(opt.symmetric && h.n_adm > 0)) predict_ranks(h, kpred.p);
        if (opt.symmetric && h.n_adm > 0) {
            // compress the canonical leaves only, then mirror
            const int64_t n = h.n_adm;
            DevBuf<int64_t> f(n, s), off(n + 1, s);
            k_canon_flag<<<grid_for(n), NT, 0, s>>>(h.ablk.p, n, f.p); note_launch();
            scan_exclusive_i64(f.p, off.p, n, off.p + n, s);
            int64_t nc = 0;
            HM_CUDA(cudaMemcpyAsync(&nc, off.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            DevBuf<uint32_t> ids(std::max<int64_t>(nc, 1), s);
            k_canon_ids<<<grid_for(n), NT, 0, s>>>(f.p, off.p, n, ids.p); note_launch();
            HM_LAUNCH("canonical leaves");
            // only the canonical leaves are compressed: predict their ranks only
            if (opt.rank_model) predict_ranks(h, kpred.p, ids.p, nc);
            compress(h, ids.p, nc, opt.rank_model ? kpred.p : nullptr);
            if (opt.rank_model) rerun_mispredicted(h);
            k_mirror<<<grid_for(n), NT, 0, s>>>(h.ablk.p, n, h.Uptr.p, h.Vptr.p, h.rank.p, h.nrej.p,
                                                h.flags.p, h.status.p); note_launch();
            HM_LAUNCH("mirror leaves");
        } else {
            compress(h, nullptr, h.n_adm, opt.rank_model ? kpred.p : nullptr);
            if (opt.rank_model) rerun_mispredicted(h);
        }
        check_status(h);
        h.stats.t_aca_ms = ta.stop_ms();
    }
    rank_stats(h);

    // product lists, near field in tile slices, U in tile slices
    {
        Timer td(s);
        // symmetric near field: store the dense leaves with tau.lo <= sigma.lo
        // only; the product applies each off-diagonal one both ways
        const Blk* dl = h.dblk.p;
        int64_t nd = h.n_dense;
        DevBuf<Blk> dcan;
        if (h.sym_near && h.n_dense > 0) {
            DevBuf<int64_t> f(h.n_dense, s), off(h.n_dense + 1, s);
            k_canon_flag<<<grid_for(h.n_dense), NT, 0, s>>>(h.dblk.p, h.n_dense, f.p); note_launch();
            scan_exclusive_i64(f.p, off.p, h.n_dense, off.p + h.n_dense, s);
            HM_CUDA(cudaMemcpyAsync(&nd, off.p + h.n_dense, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            dcan.alloc(std::max<int64_t>(nd, 1), s);
            k_canon_blocks<<<grid_for(h.n_dense), NT, 0, s>>>(h.dblk.p, f.p, off.p, h.n_dense,
                                                              dcan.p); note_launch();
            HM_LAUNCH("canonical dense leaves");
            dl = dcan.p;
        }
        mvp_build_lists(h.ablk.p, h.rank.p, h.n_adm, dl, nd, h.tile_row0.p,
                        h.tile_m.p, h.n_tiles, h.lists, s, h.sym_near);
        const MvpLists& L = h.lists;
        h.near.alloc((size_t)std::max<int64_t>(L.near_elems, 1) * near_entry_bytes(h.near_format), s);
        near_assemble(h.near_format, h.kp, h.X, dl, L.dn_ent.p,
                      L.dn_tile.p, h.tile_m.p, L.dn_desc.p, L.n_dn, h.near.p, s);
        const int esz = h.precision == HM_PREC_FP64 ? 8 : 4;
        h.ustore.alloc((size_t)std::max<int64_t>(L.u_elems, 1) * esz, s);
        mvp_relayout_u(h.precision, L, h.ablk.p, h.Uptr.p, h.tile_m.p, h.ustore.p, s);
        HM_CUDA(cudaStreamSynchronize(s));
        // the per-block U copies are no longer needed, unless mirror leaves
        // read their V from them (symmetric mode)
        if (!opt.symmetric) h.usegments.clear();
        h.stats.near_entries = L.near_elems;
        h.stats.t_dense_ms = td.stop_ms();
    }

    MvpPlan& P = h.plan;
    P.precision = h.precision;
    P.near_format = h.near_format;
    P.Ntot = Ntot;
    P.n_adm = h.n_adm;
    P.ablk = h.ablk.p;
    P.rank = h.rank.p;
    P.Uptr = h.Uptr.p;
    P.Vptr = h.Vptr.p;
    P.toff = h.lists.toff.p;
    P.t_len = h.lists.t_len;
    P.n_vitems = h.lists.n_vitems;
    P.vitems = h.lists.vitems.p;
    P.tpart_off = h.lists.tpart_off.p;
    P.tpart_len = h.lists.tpart_len;
    P.tsum_first = h.lists.tsum_first.p;
    P.tsum_count = h.lists.tsum_count.p;
    P.n_multi = h.lists.n_multi;
    P.multi = h.lists.multi.p;
    P.ustore = h.ustore.p;
    P.near = h.near.p;
    P.near_entries = h.stats.near_entries;
    P.n_tiles = h.n_tiles;
    P.max_ld = slice_ld(h.leaf);
    P.n_items = h.lists.n_items;
    P.status = h.status.p;
    P.items = h.lists.items.p;
    P.item_ptr = h.lists.item_ptr.p;
    P.tile_row0 = h.tile_row0.p;
    P.tile_m = h.tile_m.p;
    P.ucol_ptr = h.lists.ucol_ptr.p;
    P.ubase = h.lists.ubase.p;
    P.ucol_t = h.lists.ucol_t.p;
    P.ncol_ptr = h.lists.ncol_ptr.p;
    P.nbase = h.lists.nbase.p;
    P.ncol_x = h.lists.ncol_x.p;
    P.n_ucols = h.lists.n_ucols;
    P.n_ncols = h.lists.n_ncols;
    P.lr_ptr = h.lists.lr_ptr.p;
    P.lr_desc = h.lists.lr_desc.p;
    P.dn_ptr = h.lists.dn_ptr.p;
    P.dn_desc = h.lists.dn_desc.p;
    P.perm = h.perm.p;
    P.sigma2 = h.sigma2;
    P.sym_near = h.sym_near;
    P.zptr = h.lists.zptr.p;
    P.zbase = h.lists.zbase.p;
    P.zlen = h.lists.zlen.p;
    if (h.sym_near) {
        P.umid = h.lists.umid.p;
        P.n_items_b = h.lists.n_items_b;
        P.items_b = h.lists.items_b.p;
        P.item_ptr_b = h.lists.item_ptr_b.p;
        P.mirror_of = h.lists.mirror_of.p;
        P.lr_boff = h.lists.lr_boff.p;
        P.lr_pos = h.lists.lr_pos.p;
        P.lr_ecol = h.lists.lr_ecol.p;
        P.n_lr = h.lists.n_lr;
        P.big = h.lists.big.p;
        P.n_big = h.lists.n_big;
    }
    mvp_alloc_work(P, h.work, s);
    HM_CUDA(cudaStreamSynchronize(s));

    // statistics
    hm_stats& st = h.stats;
    st.n_points = Ntot;
    st.n_nodes = nn;
    st.n_adm = h.n_adm;
    st.n_dense = h.n_dense;
    st.n_tiles = h.n_tiles;
    st.depth = h.sets[0].depth;
    st.d = h.sets[0].d;
    st.precision = h.precision;
    st.near_format = h.near_format;
    const int64_t fsz = h.precision == HM_PREC_FP64 ? 8 : 4;
    st.factor_bytes = st.factor_entries * fsz;
    st.near_bytes = st.near_entries * (int64_t)near_entry_bytes(h.near_format);
    // algorithmic bytes of one product: factors + near field + x (read once
    // through the permutation) + perm + y written + the gather's column
    // multiplier indices (4 bytes per column)
    // (symmetric near field: the transposed products are written and read
    // once, 4 + 4 bytes per near column)
    const int64_t idx_bytes = (h.lists.n_ucols + h.lists.n_ncols) * 4 +
                              (h.sym_near ? 8 * h.lists.n_ncols : 0);
    st.mvp_bytes = st.factor_bytes + st.near_bytes + Ntot * (8 + 8 + 8) + idx_bytes;
    // per kernel: V^T x reads V and writes t; the gather reads U, the near
    // field, its column indices, perm and x (for sigma^2 x) and writes y
    st.mvp_vtx_bytes = (st.factor_entries - h.factor_entries_U) * fsz + h.lists.t_len * fsz;
    st.mvp_tile_bytes = h.factor_entries_U * fsz + st.near_bytes + idx_bytes;
    st.mvp_tail_bytes = Ntot * (8 + 8 + 8);   // the finish: x (sigma^2 x), perm, y
    if (h.sym_near && h.lists.umid.p) {
        // symmetric low-rank part: V^T x reads the canonical blocks' V; pass
        // A reads the canonical U and the near field and writes one float
        // per column; the tail reads those floats back (k_tmirror, the
        // finish) and streams the canonical V as the mirror slices (pass B)
        const int64_t uca = h.lists.n_ucols_canon, ucb = h.lists.n_ucols - uca;
        const int64_t nnc = h.lists.n_ncols;
        st.mvp_vtx_bytes = h.factor_entries_Vc * fsz + h.lists.t_len * fsz;
        st.mvp_tile_bytes = (h.factor_entries_U - h.factor_entries_Vc) * fsz + st.near_bytes +
                            8 * (uca + nnc);
        st.mvp_tail_bytes = h.factor_entries_Vc * fsz + 4 * ucb + 4 * (uca + nnc) + Ntot * 24;
        st.mvp_bytes = st.mvp_vtx_bytes + st.mvp_tile_bytes + st.mvp_tail_bytes;
    }
    st.t_total_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace hm
