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

// Alg. 1 on one level: classify every pair (tau, sigma) as admissible leaf,
// split (four children on the next level) or dense leaf. The classification
// is packed into one int64 per pair so that a single exclusive scan yields
// the adm offset (low 32 bits) and the dense offset (high 32 bits); the split
// offset is p - adm - dense.
// tau is a node of the row tree (lo, hi, bmin, bmax), sigma of the column
// tree (lo2, ...); the same tree for A_{phi, Y x Y}.
__global__ void k_classify(const int2* __restrict__ pairs, int64_t P, int C,
                           const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                           const double* __restrict__ bmin, const double* __restrict__ bmax,
                           const int32_t* __restrict__ lo2, const int32_t* __restrict__ hi2,
                           const double* __restrict__ bmin2, const double* __restrict__ bmax2,
                           double eta2, int adm_max, int64_t* __restrict__ flag)
{
    int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (p >= P) return;
    int2 ts = pairs[p];
    int t = ts.x, s = ts.y;
    double tmn[3], tmx[3], smn[3], smx[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        tmn[i] = bmin[(int64_t)t * 3 + i];
        tmx[i] = bmax[(int64_t)t * 3 + i];
        smn[i] = bmin2[(int64_t)s * 3 + i];
        smx[i] = bmax2[(int64_t)s * 3 + i];
    }
    bool a = admissible(tmn, tmx, smn, smx, eta2, adm_max);
    int nt = hi[t] - lo[t], ns = hi2[s] - lo2[s];
    int64_t f;
    if (a) f = 1;                          // admissible leaf
    else if (nt > C && ns > C) f = 0;      // split
    else f = 1ll << 32;                    // dense leaf
    flag[p] = f;
}

__global__ void k_emit(const int2* __restrict__ pairs, int64_t P,
                       const int64_t* __restrict__ flag, const int64_t* __restrict__ off,
                       int2* __restrict__ next, int2* __restrict__ adm, int64_t adm_base,
                       int2* __restrict__ dense, int64_t dense_base)
{
    int64_t p = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (p >= P) return;
    int64_t f = flag[p], o = off[p];
    int64_t a = o & 0xFFFFFFFFll, dn = o >> 32;
    int2 ts = pairs[p];
    if (f == 1) {
        adm[adm_base + a] = ts;
    } else if (f != 0) {
        dense[dense_base + dn] = ts;
    } else {
        int64_t sp = p - a - dn;
        int t1 = 2 * ts.x + 1, s1 = 2 * ts.y + 1;
        next[4 * sp + 0] = make_int2(t1, s1);
        next[4 * sp + 1] = make_int2(t1, s1 + 1);
        next[4 * sp + 2] = make_int2(t1 + 1, s1);
        next[4 * sp + 3] = make_int2(t1 + 1, s1 + 1);
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

// Sort a leaf list into canonical (tau.lo, sigma.lo) order.
void canonical_sort(DevBuf<int2>& leaves, int64_t n, const int32_t* lo, int64_t N,
                    const int32_t* lo2, int64_t N2, cudaStream_t s)
{
    if (n <= 1) return;
    DevBuf<uint64_t> keys(n, s);
    DevBuf<uint32_t> idx(n, s);
    k_leaf_keys<<<grid_for(n), NT, 0, s>>>(leaves.p, n, lo, lo2, N2, keys.p, idx.p); note_launch();
    HM_LAUNCH("leaf keys");
    radix_sort_u64_u32(keys.p, idx.p, n, bits_for(N + 1) + bits_for(N2 + 1), s);
    DevBuf<int2> out(n, s);
    k_gather_pairs<<<grid_for(n), NT, 0, s>>>(leaves.p, idx.p, n, out.p); note_launch();
    HM_LAUNCH("leaf gather");
    leaves = std::move(out);
}

void grow(DevBuf<int2>& buf, int64_t used, int64_t need, cudaStream_t s)
{
    if ((int64_t)buf.n >= need) return;
    int64_t cap = std::max<int64_t>(need, 2 * (int64_t)buf.n);
    DevBuf<int2> nb(cap, s);
    if (used) HM_CUDA(cudaMemcpyAsync(nb.p, buf.p, used * sizeof(int2), cudaMemcpyDeviceToDevice, s));
    buf = std::move(nb);
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

    // level-synchronous traversal (Alg. 1 via Alg. 4) from the pair of roots
    const double eta2 = eta * eta;
    DevBuf<int2> cur(1, s), nxt;
    int2 root = make_int2(0, 0);
    HM_CUDA(cudaMemcpyAsync(cur.p, &root, sizeof(int2), cudaMemcpyHostToDevice, s));
    int64_t P = 1, n_adm = 0, n_dense = 0;
    DevBuf<int64_t> tot(1, s);
    const int64_t guess = std::max<int64_t>(1024, std::max(R.N, Cs.N));
    adm.alloc(guess, s);
    dense.alloc(guess, s);
    for (int l = 0; P > 0; ++l) {
        if (l > depth) fail(HM_EOVERFLOW, "block tree deeper than the cluster trees");
        DevBuf<int64_t> flag(P, s), off(P, s);
        k_classify<<<grid_for(P), NT, 0, s>>>(cur.p, P, C, lo, hi, bn, bx, lo2, hi2, bn2, bx2,
                                              eta2, adm_max, flag.p); note_launch();
        HM_LAUNCH("classify");
        scan_exclusive_i64(flag.p, off.p, P, tot.p, s);
        int64_t h_tot = 0;
        HM_CUDA(cudaMemcpyAsync(&h_tot, tot.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        int64_t na = h_tot & 0xFFFFFFFFll, nd = h_tot >> 32, ns = P - na - nd;
        grow(adm, n_adm, n_adm + na, s);
        grow(dense, n_dense, n_dense + nd, s);
        nxt.alloc(std::max<int64_t>(4 * ns, 1), s);
        k_emit<<<grid_for(P), NT, 0, s>>>(cur.p, P, flag.p, off.p, nxt.p, adm.p, n_adm,
                                         dense.p, n_dense); note_launch();
        HM_LAUNCH("emit");
        n_adm += na;
        n_dense += nd;
        P = 4 * ns;
        std::swap(cur, nxt);
    }
    R.n_adm = n_adm;
    R.n_dense = n_dense;
    canonical_sort(adm, n_adm, lo, R.N, lo2, Cs.N, s);
    canonical_sort(dense, n_dense, lo, R.N, lo2, Cs.N, s);
}

void build_structure(const double* pts, SetStructure& S, double eta, int adm_max,
                     const DeviceCoords& X, int64_t* perm_out, uint64_t* codes_out,
                     int32_t* node_lo, int32_t* node_hi, double* bmin, double* bmax,
                     DevBuf<int2>& adm, DevBuf<int2>& dense, cudaStream_t s)
{
    build_tree(pts, S, X, perm_out, codes_out, node_lo, node_hi, bmin, bmax, s);
    traverse(S, S, eta, adm_max, node_lo, node_hi, bmin, bmax, adm, dense, s);
}

}  // namespace hm
