// hm_build.cuh -- structure builder and the kernels of the compression and
// product phases (declarations shared by the translation units).
#pragma once

#include "hm_internal.cuh"

namespace hm {

// Morton-ordered coordinates of all sets: x64[i][row] (double, zero-padded to
// three dimensions) and, for mixed precision, a hi/lo float split stored as
// six planes x32[(2i + {0,1}) * stride32 + row].
struct DeviceCoords {
    double* x64[3] = {nullptr, nullptr, nullptr};
    float* x32 = nullptr;
    int64_t stride32 = 0;
};

int tree_depth(int64_t N, int C);
int morton_bits(int d);

// Morton codes (input order) of N points; idx (may be null) receives 0..N-1;
// box receives lo[3], hi[3], scale[3].
void morton_codes(const double* pts, int64_t N, int d, uint64_t* codes, uint32_t* idx,
                  double* box, cudaStream_t s);

// Morton sort, coordinates, cluster tree, boxes, traversal and canonical leaf
// lists of one point set. pts: device (N, d) row-major. adm / dense receive
// (tau, sigma) node ids local to the set.
// One set's Morton codes, order, coordinates, cluster tree and boxes.
void build_tree(const double* pts, SetStructure& S, const DeviceCoords& X, int64_t* perm_out,
                uint64_t* codes_out, int32_t* node_lo, int32_t* node_hi, double* bmin,
                double* bmax, cudaStream_t s);
// Alg. 1 from the pair of roots of the row set R's tree and the column set
// Cs's tree (R and Cs the same set for A_{phi, Y x Y}); leaf pairs hold
// set-local node ids (tau in R's tree, sigma in Cs's), in canonical order.
// Writes R.n_adm and R.n_dense.
void traverse(SetStructure& R, const SetStructure& Cs, double eta, int adm_max,
              const int32_t* node_lo, const int32_t* node_hi, const double* bmin,
              const double* bmax, DevBuf<int2>& adm, DevBuf<int2>& dense, cudaStream_t s);
// build_tree and traverse of one set with itself.
void build_structure(const double* pts, SetStructure& S, double eta, int adm_max,
                     const DeviceCoords& X, int64_t* perm_out, uint64_t* codes_out,
                     int32_t* node_lo, int32_t* node_hi, double* bmin, double* bmax,
                     DevBuf<int2>& adm, DevBuf<int2>& dense, cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched ACA (hm_aca.cu)
// ---------------------------------------------------------------------------
struct AcaArgs {
    const Blk* blk;          // per admissible block (absolute Morton rows/cols)
    const int32_t* kres;     // reserved columns per block
    const uint64_t* Uptr;    // per block: address of U (m x kres, column-major)
    const uint64_t* Vptr;    // per block: address of V (n x kres)
    int32_t* rank;           // out: rank
    int32_t* nrej;           // out: rejected columns
    int32_t* flags;          // out: bit0 hit the reserved cap without converging
    int* status;             // out: device status word (nonzero = loop limit)
    double eps;              // aca_eps (<= 0: fixed rank)
    double aca_eta;
    double eps0;
    int k_cap;
    // Global error floor (mixed precision): the stopping tests compare with
    // max(||S_r||_F^2, m n / N_set) instead of ||S_r||_F^2, N_set the size of
    // the block's point set; null = the paper's blockwise relative test.
    const int32_t* bset;     // per block: its point set
    const int64_t* set_n;    // per set: number of points
    // Iteration limit of a block's loop; 0: k_max + n + 1 (no block needs
    // more). A smaller value is a test hook of the HM_ETIMEOUT path.
    int step_limit;
};

// Size classes of admissible blocks by d = max(m, n): class c holds the
// blocks with 2^(c+5) < d <= 2^(c+6) (class 0: d <= 64, the last class: all
// larger blocks). Classes 0-3 (d <= 512) run one warp per block, classes 4-10
// (d <= 65536) one CTA or one thread-block cluster per block with the block's
// residuals in registers, class 11 a cluster of 8 CTAs with its residuals in
// global scratch.
constexpr int ACA_NCLASS = 12;
// Rank buckets of the reservations inside a size class: bucket k holds the
// blocks with 2^(k+3) < kres <= 2^(k+4) (bucket 0 from 1, the last bucket
// unbounded); a launch of the team kernels sizes its Gram matrices for the
// bucket's largest rank (16, 32 or 64), the last bucket runs the cluster
// kernels. With the learned rank model the buckets follow the predicted
// ranks (Sec. 5.4.1's batching of similar tasks, by size and rank).
constexpr int ACA_NKB = 4;
__host__ __device__ __forceinline__ int aca_kbucket(int kres)
{
    return kres <= 16 ? 0 : kres <= 32 ? 1 : kres <= 64 ? 2 : 3;
}
__host__ __device__ __forceinline__ int aca_class_dim(int c) { return 64 << c; }
__host__ __device__ __forceinline__ int aca_class_of(int m, int n)
{
    const int d = m > n ? m : n;
    int c = 0;
    while (c < ACA_NCLASS - 1 && d > aca_class_dim(c)) ++c;
    return c;
}
// Columns block (m x n) reserves for its factors: min(k_cap, m, n) without a
// rank model; with one, its prediction kpred clamped to [1, min(k_cap, m, n)],
// and at least 32 in the size classes above 2048 rows (the few large blocks
// a model under-predicts were the long pole of the re-run phase). Every
// reservation, and every scratch sized by reservations, comes from here.
__host__ __device__ __forceinline__ int aca_reservation(int m, int n, int kcap, const int32_t* kpred,
                                                        int64_t b)
{
    const int full = kcap < (m < n ? m : n) ? kcap : (m < n ? m : n);
    if (!kpred) return full;
    int k = kpred[b] < full ? kpred[b] : full;
    if (k < 1) k = 1;
    if (aca_class_of(m, n) >= 6 && k < 32) k = full < 32 ? full : 32;
    return k;
}

// Run ACA on the blocks listed in order[0..n) (indices into the block arrays),
// all of size class cls; max_n bounds the column count of any block.
// kb is the blocks' rank bucket (aca_kbucket of every block's reservation).
void aca_run(int precision, const KernelParams& kp, const DeviceCoords& X,
             const AcaArgs& a, const uint32_t* order, int64_t n, int cls, int kb, int64_t max_n,
             cudaStream_t s);
// The same for the Matern kernel of order 1 (instantiated in its own unit).
void aca_run_k1(bool f64, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                const uint32_t* order, int64_t n, int cls, int kb, int64_t max_n, cudaStream_t s);
// Team kernels (hm_aca_team.cuh) of size class cls with Gram matrices for
// ranks up to KT; false when the class has no team shape or the shape
// control selects the cluster kernels (hm_set_aca_shape).
bool aca_team_gm(bool f64, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                 const uint32_t* order, int64_t n, int cls, int shape, int KT, cudaStream_t s);
bool aca_team_k1(bool f64, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                 const uint32_t* order, int64_t n, int cls, int shape, int KT, cudaStream_t s);
// Launch shape of the ACA of size class cls: -1 default, 0 the cluster
// kernels of hm_aca_impl.cuh, 1 .. 3 team kernel shapes (process-wide).
int aca_shape(int cls);
// The default shape of each class (the measured best).
int aca_default_shape(int cls);
// Iteration limit handed to the ACA kernels (0: none beyond k + n + 1).
int aca_step_limit();
// Test hooks of the product's bulk-copy kernels: the wait bound in ns and the
// withheld chunk (-1: none); applied to a plan by mvp_hooks.
uint64_t mvp_wait_ns();
int mvp_withhold();
void set_mvp_wait_ns(uint64_t ns);
void set_mvp_withhold(int k);
void set_aca_shape(int cls, int shape);
void set_aca_step_limit(int v);
// Test hooks of the traversal (process-wide): the first level-bound factor
// kappa (0: the default for the dimension and eta) and the number of
// traversals tried before HM_EOVERFLOW (0: 16).
void set_traversal_kappa(int64_t k);
void set_traversal_attempts(int n);
// Batching sizes (hm_set_batch_limits; 0: unlimited): reserved factor entries
// per ACA launch and work items per gather launch.
int64_t aca_batch_entries();
int64_t mvp_batch_items();
void set_batch_limits(int64_t aca_entries, int64_t gather_items);

// ---------------------------------------------------------------------------
// Product layout. The product gathers, for every row tile (a leaf of the
// cluster tree), slices of the low-rank factors U_b and of the dense blocks
// A_b restricted to the tile's rows. Both are stored tile-major: the slices a
// tile reads are contiguous and in its gather order, each slice column-major
// with the tile's row count as leading dimension.
// ---------------------------------------------------------------------------
// Leading dimension of a tile slice: the tile's rows rounded up to a
// multiple of four, so every column of a slice starts on a 16-byte boundary
// for a group of four float (or bfloat16 pair) rows; padding rows hold 0.
__host__ __device__ __forceinline__ int slice_ld(int rows) { return (rows + 3) & ~3; }

struct LrDesc {        // one (tile, admissible block) pair
    int64_t uoff;      // element offset of the slice in the tile-major U store
    int64_t toff;      // offset of t_b = V_b^T x in the t buffer
    int32_t k;         // rank (columns of the slice)
    int32_t pad;
};

struct DnDesc {        // one (tile, dense block) pair
    int64_t noff;      // element offset of the slice in the near-field store
    int64_t col0;      // first Morton column of the block
    int32_t n;         // columns of the slice
    int32_t pad;
};

// ---------------------------------------------------------------------------
// Near field (hm_near.cu)
// ---------------------------------------------------------------------------
// Evaluate the dense leaf blocks directly into their tile slices: entry e of
// the dense gather list is block ent[e].x restricted to the rows of tile
// etile[e] (offset ent[e].y in the block). In BF16X2 slices every column
// holds its slice_ld hi entries followed by its slice_ld lo entries.
void near_assemble(int near_format, const KernelParams& kp, const DeviceCoords& X,
                   const Blk* blk, const int2* ent, const int32_t* etile,
                   const int32_t* tile_m, const DnDesc* desc, int64_t n_ent, void* store,
                   cudaStream_t s);
size_t near_entry_bytes(int near_format);
// Sum over the dense leaves blk[0..n) of ||A_b||_F^2, entries in float (the
// mixed path's X.x32 coordinates); a lower bound of ||A||_F^2.
double dense_fro2(const KernelParams& kp, const DeviceCoords& X, const Blk* blk, int64_t n,
                  cudaStream_t s);

// ---------------------------------------------------------------------------
// Product (hm_mvp.cu)
// ---------------------------------------------------------------------------
struct MvpPlan {
    int precision = 0, near_format = 0;
    int64_t Ntot = 0;
    // admissible blocks
    int64_t n_adm = 0;
    const Blk* ablk = nullptr;
    const int32_t* rank = nullptr;
    const uint64_t* Uptr = nullptr;
    const uint64_t* Vptr = nullptr;
    const int64_t* toff = nullptr;     // offset of t_b in the t buffer
    int64_t t_len = 0;
    // V^T x work items: (block, column chunk)
    int64_t n_vitems = 0;
    const int2* vitems = nullptr;       // (block, chunk start)
    const int64_t* tpart_off = nullptr; // per work item: partial-sum slot
    int64_t tpart_len = 0;
    const int32_t* tsum_first = nullptr;  // per block: first work item
    const int32_t* tsum_count = nullptr;  // per block: work items
    int64_t n_multi = 0;                   // blocks with more than one item
    const int32_t* multi = nullptr;        // their ids
    // tile-major stores of the U slices and of the near field
    const void* ustore = nullptr;
    const void* near = nullptr;
    int64_t near_entries = 0;
    // flat column streams: the U slices of tile q are the ucol_ptr[q + 1] -
    // ucol_ptr[q] consecutive columns of slice_ld(rows) entries from element
    // ubase[q] of ustore, column c weighted by t[ucol_t[ucol_ptr[q] + c]];
    // its near-field slices likewise from entry nbase[q], weighted by
    // xm[ncol_x[ncol_ptr[q] + c]]
    const int64_t* ucol_ptr = nullptr;
    const int64_t* ubase = nullptr;
    const int32_t* ucol_t = nullptr;
    const int64_t* ncol_ptr = nullptr;
    const int64_t* nbase = nullptr;
    const int32_t* ncol_x = nullptr;
    int64_t n_ucols = 0, n_ncols = 0;
    // work items of the gather: item i covers columns [x, y) of tile z's
    // U-then-near column stream (items[i] = (z, x, y)); a tile's items are
    // consecutive from item_ptr[tile] and each writes max_ld partial row sums
    int64_t n_items = 0;
    const int3* items = nullptr;
    const int64_t* item_ptr = nullptr;
    int* status = nullptr;                // device status word (bounded waits)
    // bound of every mbarrier wait of the bulk-copy kernels, and a chunk that
    // their producer leaves out (-1: none); test hooks of the timeout path,
    // set per product from hm_set_test_hook
    uint64_t wait_ns = 2000000000ull;
    int withhold = -1;
    // row tiles and their gather lists (CSR over tiles)
    int64_t n_tiles = 0;
    int max_ld = 0;                       // slice_ld of the largest tile
    const int64_t* tile_row0 = nullptr;
    const int32_t* tile_m = nullptr;
    const int64_t* lr_ptr = nullptr;
    const LrDesc* lr_desc = nullptr;
    const int64_t* dn_ptr = nullptr;
    const DnDesc* dn_desc = nullptr;
    // symmetric near field: only the dense leaves with tau.lo <= sigma.lo
    // are stored; the gather also forms, for every near column of an
    // off-diagonal leaf, the transposed product (A^T x|tau)_c and writes it
    // at the column's index of the near stream into zbuf (n_ncols floats);
    // the finish adds, for tile q, records [zptr[q], zptr[q + 1]): rows
    // 0 .. zlen[r] - 1 of the tile take zbuf[zbase[r] + row]
    int sym_near = 0;
    float* zbuf = nullptr;
    const int64_t* zptr = nullptr;
    const int64_t* zbase = nullptr;
    const int32_t* zlen = nullptr;
    // symmetric low-rank part (with the symmetric near field): a tile's U
    // stream holds its canonical slices (tau.lo < sigma.lo) before its
    // mirror slices, which start at column umid[tile]. Pass A (uview 1)
    // streams the canonical slices and the near field and writes, for every
    // U column, (U^T x|tile)_c into zubuf (n_ucols floats); the mirror
    // blocks' t = U_b^T x|tau is summed from it (k_tmirror); pass B (uview
    // 2) streams the mirror slices, as items items_b / item_ptr_b whose
    // partial sums follow pass A's n_items slots.
    const int64_t* umid = nullptr;
    int uview = 0;
    float* zubuf = nullptr;
    int64_t n_items_b = 0;
    const int3* items_b = nullptr;
    const int64_t* item_ptr_b = nullptr;
    const int32_t* mirror_of = nullptr;   // per admissible block: its mirror (canonical blocks), else -1
    const int64_t* lr_boff = nullptr;     // per block: first block-major low-rank entry
    const int64_t* lr_pos = nullptr;      // block-major entry -> CSR position
    const int64_t* lr_ecol = nullptr;     // block-major entry -> its first U column
    int64_t n_lr = 0;
    const int32_t* big = nullptr;         // canonical blocks with more than 8 slices
    int64_t n_big = 0;
    // permutation and diagonal shift
    const int64_t* perm = nullptr;      // Morton row -> caller index (absolute)
    double sigma2 = 0.0;
    const double* sig_row = nullptr;    // optional per-row sigma^2 (batched sets)
};

// CUDA events around the product's kernels (when profiling), read later.
struct MvpTimer {
    struct Rec {
        cudaEvent_t e[5];
    };
    std::vector<Rec> recs;
    std::vector<Rec> pool;
    double t_total = 0, t_gather = 0, t_vtx = 0, t_tile = 0, t_tail = 0;
    int64_t count = 0;
    Rec* begin();
    void collect();   // synchronises the recorded events and sums the times
    ~MvpTimer();
};

// Work buffers of the product (xm, t, partial sums).
struct MvpWork {
    DevBuf<double> part;                  // partial row sums of the gather items
    DevBuf<double> xm64, ym64;
    DevBuf<float> xm32;
    DevBuf<double> t64, tp64;
    DevBuf<float> t32, tp32;
    // several right-hand sides (float plans), sized for MVP_NRC_MAX on first use
    DevBuf<float> xmn, tn, tpn;
    DevBuf<double> partn;
    DevBuf<float> zbuf;                   // transposed near-field products (symmetric near field)
    DevBuf<float> zubuf;                  // transposed U-slice products (symmetric low-rank part)
};

void mvp_alloc_work(const MvpPlan& P, MvpWork& W, cudaStream_t s);
// Force one launch shape of the product's gather (0 .. 4), or -1 for the
// per-device tuner; HM_EINVAL for other values.
int mvp_force_shape(int shape);
// y = H x (+ sigma^2 x) for device x, y in the caller's order.
void mvp_run(const MvpPlan& P, MvpWork& W, const double* x, double* y, int accumulate,
             cudaStream_t s, MvpTimer* timer = nullptr);
// Y = H X (+ sigma^2 X) for nrhs device right-hand sides stored one after
// another (x[r * Ntot + i]). Float plans whose slices have at most 64 rows and
// whose near field is not single bfloat16 read every stored entry once per
// group of up to MVP_NRC_MAX vectors; other plans run one product per vector.
constexpr int MVP_NRC_MAX = 16;
bool mvp_multi_fused(const MvpPlan& P);
void mvp_run_multi(const MvpPlan& P, MvpWork& W, const double* x, double* y, int nrhs,
                   int accumulate, cudaStream_t s);
// Kernels of the on-the-fly product (no stored factors or near field).
void np_gather_x(int precision, const double* x, const int64_t* perm, int64_t N, void* xm,
                 cudaStream_t s);
// Work lists of the on-the-fly low-rank part: V^T x items (block, first
// column) of 256 columns, consecutive per block from vptr[b] (h_vptr: host
// copy); apply items (tile, first entry, end entry) of at most 16 entries of
// the tile's admissible-leaf list, consecutive per tile from aptr[tile].
void np_lists(const Blk* ablk, int64_t n_adm, const int64_t* lr_ptr, int64_t n_tiles,
              DevBuf<int64_t>& vptr, DevBuf<int2>& vitems, DevBuf<int64_t>& aptr,
              DevBuf<int3>& aitems, std::vector<int64_t>& h_vptr, int64_t& n_aitems, cudaStream_t s);
// The lists of one pass q of a symmetric on-the-fly handle: its blocks are
// pblk[b0 .. b1), their V^T x items pitems[vi0 .. vi1) (block b's first at
// pfirst[b] within the pass), passid / tidx every leaf's pass and place.
struct NpSymPass {
    const int64_t* pitems = nullptr;
    const int64_t* pblk = nullptr;
    const int64_t* pfirst = nullptr;
    const int32_t* passid = nullptr;
    const int32_t* tidx = nullptr;
    int q = 0;
};
// For the admissible leaves b0 <= b < b1 (factors as left by ACA):
// t_b = V_b^T x|sigma (items vi0 .. vi1 - 1, partials in tp, sums in t), then
// every apply item's running row sums += U_b t_b in block order. With sym the
// blocks and items are those of the pass's lists (see NpSymPass) and the
// apply takes the entries of the pass's leaves in entry order.
void np_lowrank(int precision, const Blk* ablk, const int32_t* rank, const uint64_t* Uptr,
                const uint64_t* Vptr, int64_t b0, int64_t b1, const int64_t* vptr,
                const int2* vitems, int64_t vi0, int64_t vi1, const int3* aitems,
                int64_t n_aitems, const int2* lr_ent, const int32_t* tile_m, const void* xm,
                void* tp, void* t, int kcap, int ld, double* item_acc, cudaStream_t s,
                const NpSymPass* sym = nullptr);
// y_m += the apply items' row sums of every tile, in item order.
void np_apply_finish(const int64_t* aptr, const int64_t* tile_row0, const int32_t* tile_m,
                     int64_t n_tiles, int ld, const double* item_acc, double* yacc, cudaStream_t s);
// y_m += A_b x|sigma for every dense leaf, entries evaluated on the fly, over
// the gather's work items (runs of a tile's near-field column stream); part
// holds n_items * max_ld partial row sums.
void np_near(int precision, const KernelParams& kp, const DeviceCoords& X, const int3* items,
             int64_t n_items, const int64_t* item_ptr, const int64_t* ucol_ptr,
             const int64_t* ncol_ptr, const int32_t* ncol_x, const int64_t* tile_row0,
             const int32_t* tile_m, int64_t n_tiles, int max_ld, const void* xm, double* part,
             double* yacc, cudaStream_t s);
// y[perm[i]] = y_m[i] + sigma^2 x[perm[i]] (or +=).
void np_finish(const int64_t* perm, const double* sig_row, double sigma2, int64_t N,
               const double* yacc, const double* x, double* y, int accumulate, cudaStream_t s);
// Build the gather lists of the plan (CSR by tile).
struct MvpLists {
    DevBuf<int64_t> lr_ptr, dn_ptr;
    DevBuf<int2> lr_ent, dn_ent;          // (block, row offset of the tile)
    DevBuf<int32_t> lr_tile, dn_tile;     // tile of every entry
    DevBuf<LrDesc> lr_desc;
    DevBuf<DnDesc> dn_desc;
    DevBuf<int2> vitems;
    DevBuf<int64_t> tpart_off, toff;
    DevBuf<int32_t> tsum_first, tsum_count, multi;
    DevBuf<int64_t> ucol_ptr, ubase, ncol_ptr, nbase;   // flat column streams
    DevBuf<int32_t> ucol_t, ncol_x;
    int64_t n_ucols = 0, n_ncols = 0;
    DevBuf<int3> items;                      // gather work items
    DevBuf<int64_t> item_ptr;
    int64_t n_items = 0;
    int64_t n_tiles = 0, n_vitems = 0, tpart_len = 0, t_len = 0, n_multi = 0;
    int64_t n_lr = 0, n_dn = 0, u_elems = 0, near_elems = 0;
    // symmetric near field (sym_near): transposed-product records per tile
    int sym_near = 0;
    DevBuf<int64_t> zptr, zbase;
    DevBuf<int32_t> zlen;
    int64_t n_zrec = 0, n_zcols = 0;
    // symmetric low-rank part (with sym_near): see MvpPlan
    DevBuf<int64_t> umid, item_ptr_b, lr_boff, lr_pos, lr_ecol;
    DevBuf<int3> items_b;
    DevBuf<int32_t> mirror_of, big;
    int64_t n_items_b = 0, n_big = 0;
    int64_t u_elems_canon = 0;   // elements of the canonical slices
    int64_t n_ucols_canon = 0;   // U columns of the canonical slices
};
// dblk: the dense leaves to store; with sym_near they are the canonical ones
// (row0 <= col0) and the lists also get the transposed-product records.
void mvp_build_lists(const Blk* ablk, const int32_t* rank, int64_t n_adm, const Blk* dblk,
                     int64_t n_dense, const int64_t* leaf_row0, const int32_t* leaf_m,
                     int64_t n_tiles, MvpLists& L, cudaStream_t s, int sym_near = 0);
// Copy every block's U rows of every tile it covers into the tile-major store.
void mvp_relayout_u(int precision, const MvpLists& L, const Blk* ablk, const uint64_t* Uptr,
                    const int32_t* tile_m, void* ustore, cudaStream_t s);

}  // namespace hm
