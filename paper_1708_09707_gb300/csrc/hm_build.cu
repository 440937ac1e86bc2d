// hm_build.cu -- structure of the H-matrix on the device: global box, Morton
// codes (Alg. 6), radix sort (Sec. 4.4), Morton-ordered coordinates
// (Sec. 5.1), cluster-tree ranges and bounding boxes (Sec. 2.1-2.2, 5.3),
// level-synchronous block-tree traversal with the admissibility test
// (Alg. 1 evaluated level by level as in Alg. 4) and the canonical order of
// the two leaf lists (Sec. 5.4, Fig. workQueue).
//
// Floating-point decisions that fix integers (the fixed-point Morton
// coordinate, the admissibility test) are written with explicit
// round-to-nearest intrinsics so that the compiler cannot contract them into
// fused multiply-adds: the sequence of IEEE operations is the one stated in
// the comments.
#include <atomic>
#include <cmath>

#include "hm_build.cuh"

namespace hm {

namespace {

constexpr int NT = 256;

// --------------------------------------------------------------------------
// Global bounding box of the input points (row-major (N, d)) and the
// per-dimension Morton scale s_i = 2^b / (hi_i - lo_i) (0 for a flat
// dimension). Also flags non-finite coordinates.
// --------------------------------------------------------------------------
__global__ void k_box_partial(const double* __restrict__ pts, int64_t N, int d,
                              double* __restrict__ part, int* __restrict__ bad)
{
    __shared__ double smin[3][NT], smax[3][NT];
    double lo[3] = {INFINITY, INFINITY, INFINITY};
    double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int nonfinite = 0;
    for (int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * NT) {
        for (int i = 0; i < d; ++i) {
            double x = pts[p * d + i];
            if (!isfinite(x)) nonfinite = 1;
            lo[i] = fmin(lo[i], x);
            hi[i] = fmax(hi[i], x);
        }
    }
    if (nonfinite) atomicOr(bad, 1);
    for (int i = 0; i < 3; ++i) {
        smin[i][threadIdx.x] = lo[i];
        smax[i][threadIdx.x] = hi[i];
    }
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int i = 0; i < 3; ++i) {
                smin[i][threadIdx.x] = fmin(smin[i][threadIdx.x], smin[i][threadIdx.x + o]);
                smax[i][threadIdx.x] = fmax(smax[i][threadIdx.x], smax[i][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int i = 0; i < 3; ++i) {
            part[blockIdx.x * 6 + i] = smin[i][0];
            part[blockIdx.x * 6 + 3 + i] = smax[i][0];
        }
}

// box[0..2] = lo, box[3..5] = hi, box[6..8] = scale
__global__ void k_box_final(const double* __restrict__ part, int nb, int d, int bits,
                            double* __restrict__ box)
{
    if (threadIdx.x != 0) return;
    for (int i = 0; i < 3; ++i) {
        double lo = INFINITY, hi = -INFINITY;
        for (int b = 0; b < nb; ++b) {
            lo = fmin(lo, part[b * 6 + i]);
            hi = fmax(hi, part[b * 6 + 3 + i]);
        }
        if (i >= d) lo = hi = 0.0;
        box[i] = lo;
        box[3 + i] = hi;
        // s_i = 2^b / (hi - lo): IEEE division, as on the host
        box[6 + i] = (hi > lo) ? __ddiv_rn(ldexp(1.0, bits), __dsub_rn(hi, lo)) : 0.0;
    }
}

// Spread the low bits of x so that consecutive bits land d apart.
__device__ __forceinline__ uint64_t spread2(uint64_t x)
{
    x &= 0xFFFFFFFFull;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

__device__ __forceinline__ uint64_t spread3(uint64_t x)
{
    x &= 0x1FFFFFull;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Alg. 6: fixed point q_i = min(floor((x_i - lo_i) * s_i), 2^b - 1), then the
// bits of dimension i are stretched d apart and interleaved with dimension 0
// most significant.
__global__ void k_morton(const double* __restrict__ pts, int64_t N, int d, int bits,
                         const double* __restrict__ box, uint64_t* __restrict__ codes,
                         uint32_t* __restrict__ idx)
{
    int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (p >= N) return;
    const uint64_t qmax = (bits >= 64) ? ~0ull : ((1ull << bits) - 1ull);
    uint64_t q[3] = {0, 0, 0};
    for (int i = 0; i < d; ++i) {
        double f = floor(__dmul_rn(__dsub_rn(pts[p * d + i], box[i]), box[6 + i]));
        q[i] = (f >= (double)qmax) ? qmax : (uint64_t)f;
    }
    uint64_t c;
    if (d == 1) c = q[0];
    else if (d == 2) c = (spread2(q[0]) << 1) | spread2(q[1]);
    else c = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    codes[p] = c;
    if (idx) idx[p] = (uint32_t)p;
}

// Morton-ordered coordinates (zero-padded to 3) and the permutation.
__global__ void k_permute(const double* __restrict__ pts, int64_t N, int d,
                          const uint32_t* __restrict__ perm, double* __restrict__ X0,
                          double* __restrict__ X1, double* __restrict__ X2,
                          float* __restrict__ F, int64_t fstride,
                          int64_t* __restrict__ perm_out)
{
    int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (j >= N) return;
    int64_t src = perm[j];
    double x[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < d; ++i) x[i] = pts[src * d + i];
    X0[j] = x[0];
    X1[j] = x[1];
    X2[j] = x[2];
    if (F) {
        // hi/lo float split: x = hi + lo to about 2^-48 relative
        for (int i = 0; i < 3; ++i) {
            float h = __double2float_rn(x[i]);
            float l = __double2float_rn(x[i] - (double)h);
            F[(2 * i) * fstride + j] = h;
            F[(2 * i + 1) * fstride + j] = l;
        }
    }
    perm_out[j] = src;
}

// Cluster tree: node v (heap numbering) covers [lo, hi); halving rule with the
// left child taking floor(size/2); a node exists iff its parent has > C.
__global__ void k_tree_ranges(int64_t n_nodes, int64_t N, int C,
                              int32_t* __restrict__ lo_out, int32_t* __restrict__ hi_out)
{
    int64_t v = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (v >= n_nodes) return;
    // path from the root: bits of (v+1) below its leading one
    uint64_t key = (uint64_t)v + 1;
    int lev = 63 - __clzll(key);
    int64_t lo = 0, hi = N;
    bool ok = true;
    for (int b = lev - 1; b >= 0; --b) {
        if (hi - lo <= C) {
            ok = false;
            break;
        }
        int64_t mid = lo + (hi - lo) / 2;
        if ((key >> b) & 1) lo = mid;
        else hi = mid;
    }
    lo_out[v] = ok ? (int32_t)lo : -1;
    hi_out[v] = ok ? (int32_t)hi : -1;
}

// Bounding boxes of the nodes of one level: internal nodes merge their two
// children (computed by the previous launch), leaves reduce their range. One
// warp per node. Min and max are exact, so the result does not depend on the
// order of the reduction.
__global__ void k_bbox_level(int64_t first, int64_t count, int C,
                             const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                             const double* __restrict__ X0, const double* __restrict__ X1,
                             const double* __restrict__ X2, double* __restrict__ bmin,
                             double* __restrict__ bmax)
{
    int64_t w = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= count) return;
    int64_t v = first + w;
    int a = lo[v], b = hi[v];
    if (a < 0) return;
    if (b - a > C) {
        if (lane < 3) {
            int64_t c1 = 2 * v + 1, c2 = 2 * v + 2;
            bmin[v * 3 + lane] = fmin(bmin[c1 * 3 + lane], bmin[c2 * 3 + lane]);
            bmax[v * 3 + lane] = fmax(bmax[c1 * 3 + lane], bmax[c2 * 3 + lane]);
        }
        return;
    }
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = a + lane; j < b; j += 32) {
        double x0 = X0[j], x1 = X1[j], x2 = X2[j];
        mn[0] = fmin(mn[0], x0); mx[0] = fmax(mx[0], x0);
        mn[1] = fmin(mn[1], x1); mx[1] = fmax(mx[1], x1);
        mn[2] = fmin(mn[2], x2); mx[2] = fmax(mx[2], x2);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int i = 0; i < 3; ++i) {
            mn[i] = fmin(mn[i], __shfl_xor_sync(0xffffffffu, mn[i], o));
            mx[i] = fmax(mx[i], __shfl_xor_sync(0xffffffffu, mx[i], o));
        }
    if (lane < 3) {
        bmin[v * 3 + lane] = mn[lane];
        bmax[v * 3 + lane] = mx[lane];
    }
}

// Eq. (admissibilityCondition) in squared form with a fixed operation order:
// D2 = sum_i (b_i - a_i)^2, G2 = sum_i (g1^2 + g2^2), g1 = max(0, a_t - b_s),
// g2 = max(0, a_s - b_t); admissible iff min (or max) {D2_t, D2_s} <= eta2 G2.
__device__ __forceinline__ bool admissible(const double* tmn, const double* tmx,
                                           const double* smn, const double* smx,
                                           double eta2, int adm_max)
{
    double Dt = 0.0, Ds = 0.0, G2 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double et = __dsub_rn(tmx[i], tmn[i]);
        double es = __dsub_rn(smx[i], smn[i]);
        Dt = __dadd_rn(Dt, __dmul_rn(et, et));
        Ds = __dadd_rn(Ds, __dmul_rn(es, es));
        double g1 = __dsub_rn(tmn[i], smx[i]);
        double g2 = __dsub_rn(smn[i], tmx[i]);
        if (g1 < 0.0) g1 = 0.0;
        if (g2 < 0.0) g2 = 0.0;
        G2 = __dadd_rn(G2, __dadd_rn(__dmul_rn(g1, g1), __dmul_rn(g2, g2)));
    }
    double D = adm_max ? (Dt > Ds ? Dt : Ds) : (Dt < Ds ? Dt : Ds);
    return D <= __dmul_rn(eta2, G2);
}

// Alg. 1 on one level (Alg. 4's level-synchronous form): classify every
// pair (tau, sigma) as admissible leaf, split (four children on the next
// level) or dense leaf. The classification is packed into one int64 per pair
// so that a single exclusive scan yields the adm offset (low 32 bits) and the
// dense offset (high 32 bits); the split offset is p - adm - dense.
// tau is a node of the row tree (lo, hi, bmin, bmax), sigma of the column
// tree (lo2, ...); the same tree for A_{phi, Y x Y}.
//
// The level's pair count stays on the device: cnt = {P, admissible leaves so
// far, dense leaves so far}. The grids are sized for the level's bound and
// stride over the P pairs, so no launch waits for the host to learn P.
__global__ void k_classify(const int2* __restrict__ pairs, const int64_t* __restrict__ cnt,
                           int64_t B, int C, const int32_t* __restrict__ lo,
                           const int32_t* __restrict__ hi, const double* __restrict__ bmin,
                           const double* __restrict__ bmax, const int32_t* __restrict__ lo2,
                           const int32_t* __restrict__ hi2, const double* __restrict__ bmin2,
                           const double* __restrict__ bmax2, double eta2, int adm_max,
                           int64_t* __restrict__ flag)
{
    const int64_t P = cnt[0] < B ? cnt[0] : B;
    for (int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * NT) {
        const int2 ts = pairs[p];
        const int t = ts.x, s = ts.y;
        double tmn[3], tmx[3], smn[3], smx[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            tmn[i] = bmin[(int64_t)t * 3 + i];
            tmx[i] = bmax[(int64_t)t * 3 + i];
            smn[i] = bmin2[(int64_t)s * 3 + i];
            smx[i] = bmax2[(int64_t)s * 3 + i];
        }
        const bool a = admissible(tmn, tmx, smn, smx, eta2, adm_max);
        const int nt = hi[t] - lo[t], ns = hi2[s] - lo2[s];
        int64_t f;
        if (a) f = 1;                          // admissible leaf
        else if (nt > C && ns > C) f = 0;      // split
        else f = 1ll << 32;                    // dense leaf
        flag[p] = f;
    }
}

// Writes the level's leaves into one arena of BL pairs, admissible leaves
// from the front and dense leaves from the back, and its splits' children
// into next (at most Bnext pairs). Children that would pass Bnext are not
// written; k_level_advance then stops the traversal and raises the overflow
// word.
__global__ void k_emit(const int2* __restrict__ pairs, int64_t B, const int64_t* __restrict__ flag,
                       const int64_t* __restrict__ off, const int64_t* __restrict__ cnt,
                       int2* __restrict__ next, int64_t Bnext, int2* __restrict__ leaves,
                       int64_t BL)
{
    const int64_t P = cnt[0] < B ? cnt[0] : B;
    const int64_t adm0 = cnt[1], dense0 = cnt[2];
    for (int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * NT) {
        const int64_t f = flag[p], o = off[p];
        const int64_t a = o & 0xFFFFFFFFll, dn = o >> 32;
        const int2 ts = pairs[p];
        if (f == 1) {
            const int64_t at = adm0 + a;
            if (at < BL) leaves[at] = ts;
        } else if (f != 0) {
            const int64_t at = BL - 1 - (dense0 + dn);
            if (at >= 0) leaves[at] = ts;
        } else {
            const int64_t sp = p - a - dn;
            if (4 * sp + 3 >= Bnext) continue;
            const int t1 = 2 * ts.x + 1, s1 = 2 * ts.y + 1;
            next[4 * sp + 0] = make_int2(t1, s1);
            next[4 * sp + 1] = make_int2(t1, s1 + 1);
            next[4 * sp + 2] = make_int2(t1 + 1, s1);
            next[4 * sp + 3] = make_int2(t1 + 1, s1 + 1);
        }
    }
}

// After a level: the leaf counts and the next level's pair count; a next
// level above its bound (or leaves above the arena) sets *ovf and ends the
// traversal (P = 0), so that no later launch reads a pair never written.
__global__ void k_level_advance(const int64_t* __restrict__ tot, int64_t* __restrict__ cnt,
                                int64_t Bnext, int64_t BL, int* __restrict__ ovf)
{
    const int64_t t = *tot;
    const int64_t P = cnt[0];
    const int64_t na = t & 0xFFFFFFFFll, nd = t >> 32;
    const int64_t ns = P - na - nd;
    cnt[1] += na;
    cnt[2] += nd;
    if (4 * ns > Bnext || cnt[1] + cnt[2] > BL) {
        *ovf = 1;
        cnt[0] = 0;
    } else {
        cnt[0] = 4 * ns;
    }
}

// Canonical leaf order key: tau.lo * N2 + sigma.lo (tau.lo in the row tree,
// sigma.lo in the column tree, N2 the column set's size).
__global__ void k_leaf_keys(const int2* __restrict__ leaves, int64_t n,
                            const int32_t* __restrict__ lo, const int32_t* __restrict__ lo2,
                            int64_t N2, uint64_t* __restrict__ keys, uint32_t* __restrict__ idx)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b >= n) return;
    int2 ts = leaves[b];
    keys[b] = (uint64_t)lo[ts.x] * (uint64_t)N2 + (uint64_t)lo2[ts.y];
    idx[b] = (uint32_t)b;
}

__global__ void k_gather_pairs(const int2* __restrict__ in, const uint32_t* __restrict__ idx,
                               int64_t n, int2* __restrict__ out)
{
    int64_t b = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (b < n) out[b] = in[idx[b]];
}

inline unsigned grid_for(int64_t n) { return (unsigned)ceil_div(n, NT); }

int bits_for(int64_t n)
{
    int b = 0;
    while ((1ll << b) < n) ++b;
    return b;
}

// Sort n leaf pairs (device, in) into canonical (tau.lo, sigma.lo) order in
// out (allocated here, n pairs).
void canonical_sort(const int2* in, int64_t n, DevBuf<int2>& out, const int32_t* lo, int64_t N,
                    const int32_t* lo2, int64_t N2, cudaStream_t s)
{
    out.alloc(std::max<int64_t>(n, 1), s);
    if (n == 0) return;
    if (n == 1) {
        HM_CUDA(cudaMemcpyAsync(out.p, in, sizeof(int2), cudaMemcpyDeviceToDevice, s));
        return;
    }
    DevBuf<uint64_t> keys(n, s);
    DevBuf<uint32_t> idx(n, s);
    k_leaf_keys<<<grid_for(n), NT, 0, s>>>(in, n, lo, lo2, N2, keys.p, idx.p); note_launch();
    HM_LAUNCH("leaf keys");
    radix_sort_u64_u32(keys.p, idx.p, n, bits_for(N + 1) + bits_for(N2 + 1), s);
    k_gather_pairs<<<grid_for(n), NT, 0, s>>>(in, idx.p, n, out.p); note_launch();
    HM_LAUNCH("leaf gather");
}

// Level bounds of the traversal: level l of the block tree holds at most
// min(4^l, kappa 2^l) pairs. A cluster of level l meets a bounded number of
// clusters of its level that it is not yet separated from (Sec. 2.2: the
// admissibility condition compares diameter and distance), about 2^l of
// them per unit of kappa; kappa grows with the dimension and with 1 / eta.
std::atomic<int64_t> g_trav_kappa{0};
std::atomic<int> g_trav_attempts{0};

int64_t default_kappa(int d, double eta)
{
    int64_t k = d <= 1 ? 16 : d == 2 ? 256 : 1024;
    if (eta < 1.0) {
        const double f = std::ceil(1.0 / eta);
        k = (int64_t)std::min(std::pow(f, (double)std::max(d, 1)) * (double)k, 1048576.0);
    }
    return k;
}

}  // namespace

int tree_depth(int64_t N, int C)
{
    int depth = 0;
    int64_t sz = N;
    while (sz > C) {
        sz = sz - sz / 2;
        depth++;
    }
    return depth;
}

int morton_bits(int d) { return d == 1 ? 32 : (d == 2 ? 32 : 21); }

void morton_codes(const double* pts, int64_t N, int d, uint64_t* codes, uint32_t* idx,
                  double* box, cudaStream_t s)
{
    int nb = (int)std::min<int64_t>(ceil_div(N, NT), 4 * (int64_t)num_sms());
    if (nb < 1) nb = 1;
    DevBuf<double> part((size_t)nb * 6, s);
    DevBuf<int> bad(1, s);
    HM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    k_box_partial<<<nb, NT, 0, s>>>(pts, N, d, part.p, bad.p); note_launch();
    k_box_final<<<1, 32, 0, s>>>(part.p, nb, d, morton_bits(d), box); note_launch();
    k_morton<<<grid_for(N), NT, 0, s>>>(pts, N, d, morton_bits(d), box, codes, idx); note_launch();
    HM_LAUNCH("morton");
    int hbad = 0;
    HM_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    if (hbad) fail(HM_EINVAL, "non-finite point coordinate");
}

void build_tree(const double* pts, SetStructure& S, const DeviceCoords& X, int64_t* perm_out,
                uint64_t* codes_out, int32_t* node_lo, int32_t* node_hi, double* bmin,
                double* bmax, cudaStream_t s)
{
    const int64_t N = S.N;
    const int d = S.d, C = S.C;
    S.depth = tree_depth(N, C);
    S.n_nodes = (2ll << S.depth) - 1;

    // Morton codes and the stable sort (Sec. 4.4)
    DevBuf<uint64_t> codes(N, s);
    DevBuf<uint32_t> idx(N, s);
    DevBuf<double> box(9, s);
    morton_codes(pts, N, d, codes.p, idx.p, box.p, s);
    if (codes_out)
        HM_CUDA(cudaMemcpyAsync(codes_out, codes.p, N * sizeof(uint64_t),
                                cudaMemcpyDeviceToDevice, s));
    radix_sort_u64_u32(codes.p, idx.p, N, d * morton_bits(d), s);

    // Morton-ordered coordinates (Sec. 5.1, point_set)
    const int64_t r0 = S.row0;
    k_permute<<<grid_for(N), NT, 0, s>>>(pts, N, d, idx.p, X.x64[0] + r0, X.x64[1] + r0,
                                        X.x64[2] + r0, X.x32 ? X.x32 + r0 : nullptr,
                                        X.stride32, perm_out + r0); note_launch();
    HM_LAUNCH("permute");

    // cluster tree and bounding boxes, bottom-up one level per launch
    int32_t* lo = node_lo + S.node0;
    int32_t* hi = node_hi + S.node0;
    double* bn = bmin + S.node0 * 3;
    double* bx = bmax + S.node0 * 3;
    k_tree_ranges<<<grid_for(S.n_nodes), NT, 0, s>>>(S.n_nodes, N, C, lo, hi); note_launch();
    HM_LAUNCH("tree ranges");
    for (int l = S.depth; l >= 0; --l) {
        int64_t first = (1ll << l) - 1, count = 1ll << l;
        k_bbox_level<<<grid_for(count * 32), NT, 0, s>>>(first, count, C, lo, hi,
                                                         X.x64[0] + r0, X.x64[1] + r0,
                                                         X.x64[2] + r0, bn, bx); note_launch();
    }
    HM_LAUNCH("bbox");
}

void traverse(SetStructure& R, const SetStructure& Cs, double eta, int adm_max,
              const int32_t* node_lo, const int32_t* node_hi, const double* bmin,
              const double* bmax, DevBuf<int2>& adm, DevBuf<int2>& dense, cudaStream_t s)
{
    const int C = R.C;
    const int32_t* lo = node_lo + R.node0;
    const int32_t* hi = node_hi + R.node0;
    const double* bn = bmin + R.node0 * 3;
    const double* bx = bmax + R.node0 * 3;
    const int32_t* lo2 = node_lo + Cs.node0;
    const int32_t* hi2 = node_hi + Cs.node0;
    const double* bn2 = bmin + Cs.node0 * 3;
    const double* bx2 = bmax + Cs.node0 * 3;
    const int depth = std::max(R.depth, Cs.depth);

    // level-synchronous traversal (Alg. 1 via Alg. 4) from the pair of roots,
    // every count kept on the device: the host reads the leaf counts once,
    // after the last level, and runs the traversal again with twice the
    // level bounds if a level did not fit
    const double eta2 = eta * eta;
    const int L = depth + 1;
    const int d = std::max(R.d, Cs.d);
    int64_t kappa = g_trav_kappa.load() > 0 ? g_trav_kappa.load() : default_kappa(d, eta);
    const int attempts = g_trav_attempts.load() > 0 ? g_trav_attempts.load() : 16;
    const int gmax = 8 * num_sms();
    for (int attempt = 0;; ++attempt) {
        if (attempt >= attempts)
            fail(HM_EOVERFLOW, "block-tree level bounds still too small after " +
                                   std::to_string(attempts) + " traversals");
        std::vector<int64_t> bound(L + 1);
        int64_t bmax_l = 1, bsum = 0;
        for (int l = 0; l <= L; ++l) {
            const int64_t full = l < 31 ? (1ll << (2 * l)) : (1ll << 62);
            const int64_t geo = (l < 40 && kappa < (1ll << 20)) ? kappa << l : (1ll << 62);
            bound[l] = std::max<int64_t>(1, std::min(full, geo));
            if (l < L) {
                bmax_l = std::max(bmax_l, bound[l]);
                bsum += bound[l];
            }
        }
        bmax_l = std::max(bmax_l, bound[L]);
        DevBuf<int2> cur(bmax_l, s), nxt(bmax_l, s), leaves(bsum, s);
        DevBuf<int64_t> flag(bmax_l, s), off(bmax_l, s), tot(1, s), cnt(3, s);
        DevBuf<int> ovf(1, s);
        const int2 root = make_int2(0, 0);
        const int64_t c0[3] = {1, 0, 0};
        HM_CUDA(cudaMemcpyAsync(cur.p, &root, sizeof(int2), cudaMemcpyHostToDevice, s));
        HM_CUDA(cudaMemcpyAsync(cnt.p, c0, sizeof(c0), cudaMemcpyHostToDevice, s));
        HM_CUDA(cudaMemsetAsync(ovf.p, 0, sizeof(int), s));
        for (int l = 0; l < L; ++l) {
            const int64_t B = bound[l];
            const unsigned g = (unsigned)std::min<int64_t>(grid_for(B), gmax);
            k_classify<<<g, NT, 0, s>>>(cur.p, cnt.p, B, C, lo, hi, bn, bx, lo2, hi2, bn2, bx2,
                                        eta2, adm_max, flag.p); note_launch();
            HM_LAUNCH("classify");
            scan_exclusive_i64_dev(flag.p, off.p, cnt.p, B, tot.p, s);
            k_emit<<<g, NT, 0, s>>>(cur.p, B, flag.p, off.p, cnt.p, nxt.p, bound[l + 1],
                                    leaves.p, bsum); note_launch();
            k_level_advance<<<1, 1, 0, s>>>(tot.p, cnt.p, bound[l + 1], bsum, ovf.p); note_launch();
            HM_LAUNCH("emit");
            std::swap(cur, nxt);
        }
        int64_t hc[3] = {0, 0, 0};
        int hovf = 0;
        HM_CUDA(cudaMemcpyAsync(hc, cnt.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(&hovf, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        if (hovf) {
            kappa *= 2;
            continue;
        }
        if (hc[0] != 0) fail(HM_EOVERFLOW, "block tree deeper than the cluster trees");
        R.n_adm = hc[1];
        R.n_dense = hc[2];
        R.traversal_reruns = attempt;
        // admissible leaves at the front of the arena, dense leaves at its back
        canonical_sort(leaves.p, R.n_adm, adm, lo, R.N, lo2, Cs.N, s);
        canonical_sort(leaves.p + (bsum - R.n_dense), R.n_dense, dense, lo, R.N, lo2, Cs.N, s);
        return;                            // the arena's free is stream-ordered
    }
}

void set_traversal_kappa(int64_t k) { g_trav_kappa = k; }
void set_traversal_attempts(int n) { g_trav_attempts = n; }

void build_structure(const double* pts, SetStructure& S, double eta, int adm_max,
                     const DeviceCoords& X, int64_t* perm_out, uint64_t* codes_out,
                     int32_t* node_lo, int32_t* node_hi, double* bmin, double* bmax,
                     DevBuf<int2>& adm, DevBuf<int2>& dense, cudaStream_t s)
{
    build_tree(pts, S, X, perm_out, codes_out, node_lo, node_hi, bmin, bmax, s);
    traverse(S, S, eta, adm_max, node_lo, node_hi, bmin, bmax, adm, dense, s);
}

}  // namespace hm
