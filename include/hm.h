/*
 * hm.h -- C-ABI of libhm.so: GB300 (sm_103a) H-matrix build and H-matrix-vector
 * product for kernel matrices A_{phi,Y x Y} (optionally + sigma^2 I), after
 * P. Zaspel, "Algorithmic patterns for H-matrices on many-core processors"
 * (arXiv 1708.09707).
 *
 * Conventions for every entry point:
 *  - Pointers may be host (pageable or pinned) or device memory of the current
 *    CUDA device; the library tells them apart with cudaPointerGetAttributes.
 *    Host inputs are copied in, host outputs copied out before return.
 *  - Functions returning int give HM_OK (0) or a negative HM_E* code and never
 *    abort the process; hm_last_error() describes the last failure of the
 *    calling thread. No kernel traps: device-side failures (loop limits) set a
 *    status word that the host turns into HM_ETIMEOUT.
 *  - The caller keeps ownership of every pointer it passes; the library keeps
 *    no reference to caller memory after a call returns. The handle owns all
 *    device memory it allocates until hm_free.
 *  - Work is enqueued on the handle's stream (hm_options.stream, default the
 *    legacy default stream). Functions that return data to host memory, or
 *    read sizes back, synchronise that stream.
 *  - All floating-point inputs are IEEE double; the arithmetic used inside is
 *    set by hm_options.precision.
 */
#ifndef HM_H
#define HM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Kernel functions phi(y, y') of r = |y - y'|, params[0] = length scale l > 0:
 *   HM_GAUSSIAN:  exp(-r^2 / l^2)           (Sec. 6.2 uses l = 1)
 *   HM_MATERN32:  (1 + sqrt3 r / l) exp(-sqrt3 r / l)
 *   HM_MATERN_K1: s K_1(s), s = r / l: the Matern kernel of Sec. 6.2 with
 *                 beta - d/2 = 1 (K_1 the modified Bessel function of the
 *                 second kind of order 1), normalised to phi(0) = 1; the
 *                 paper's form is this times 1 / (2^(beta-1) Gamma(beta)),
 *                 1/2 for d = 2 and 0.26596 for d = 3, a constant factor of
 *                 the whole matrix that leaves blocks, ranks and relative
 *                 errors unchanged.
 * params[1] = sigma^2 >= 0 is added on the diagonal by the product (Sec. 1,
 * the GPR / kernel ridge regression system A + sigma^2 I). */
enum { HM_GAUSSIAN = 0, HM_MATERN32 = 1, HM_MATERN_K1 = 2 };

enum {
    HM_OK = 0,
    HM_EINVAL = -1,     /* bad argument (sizes, parameters, non-finite input) */
    HM_ENOMEM = -2,     /* device allocation failed */
    HM_EOVERFLOW = -3,  /* an internal bound was exceeded and could not grow */
    HM_ECUDA = -4,      /* a CUDA runtime call failed */
    HM_ETIMEOUT = -5,   /* a device loop hit its iteration limit */
    HM_ENOTSUP = -6     /* option combination not supported */
};

/* Arithmetic of the build and the product. */
enum {
    HM_PREC_FP64 = 0,   /* everything in double precision */
    HM_PREC_MIXED = 1   /* FP32 kernel evaluation, ACA and factors; FP64 ACA
                           stopping test; near field per near_format; FP32
                           products with compensated accumulation */
};

/* Storage of the near-field (inadmissible) leaf blocks. */
enum {
    HM_NEAR_AUTO = 0,   /* FP64 for HM_PREC_FP64, BF16X2 for HM_PREC_MIXED */
    HM_NEAR_FP64 = 1,
    HM_NEAR_FP32 = 2,
    HM_NEAR_BF16X2 = 3, /* hi + lo bfloat16 pair per entry (about 16 bits) */
    HM_NEAR_BF16 = 4    /* single bfloat16 (8 bits; about 1e-3 per entry) */
};

typedef struct hm_options {
    int precision;        /* HM_PREC_*, default HM_PREC_FP64 */
    int near_format;      /* HM_NEAR_*, default HM_NEAR_AUTO */
    int adm_max;          /* 0: min{diam} <= eta dist (paper), 1: max{diam} */
    int k_cap;            /* ACA rank cap, default 64; fixed rank when aca_eps<=0 */
    double aca_eta;       /* eta of the ACA stopping rule, default 0 */
    double eps0;          /* column rejection threshold, <=0: 1e-14 (FP64) / 1e-6 */
    int accumulate;       /* hm_matvec: 0 overwrite y, 1 y += H x */
    int rank_model;       /* 1: size factor storage by the learned rank model */
    const float* rank_model_theta; /* 4801 FP32 weights (host or device), or NULL */
    double scratch_gb;    /* bound on ACA scratch per pass, <=0: automatic */
    void* stream;         /* cudaStream_t, NULL = legacy default stream */
    int profile;          /* 1: time every product kernel with CUDA events on
                             the launching stream (read by hm_get_stats);
                             2: as 1, and run the ACA size classes one after
                             another instead of concurrently, so that
                             t_aca_class_ms holds each class's own duration */
    int structure_only;   /* 1: stop after the cluster tree and the leaf lists
                             (no ACA, no near field; hm_matvec is refused) */
    int symmetric;        /* 1: use phi(y, y') = phi(y', y): compress only the
                             admissible leaves (tau, sigma) with tau.lo <=
                             sigma.lo; each mirror leaf (sigma, tau) takes the
                             same factors with U and V exchanged, so the
                             H-matrix is symmetric and ACA does half the work.
                             2: as 1, and store the dense leaves with tau.lo <=
                             sigma.lo only: the product applies each
                             off-diagonal one to both its rows (A x|sigma) and
                             its mirror's rows (A^T x|tau, through a buffer of
                             one value per stored column added in a fixed
                             order), so the near field's bytes about halve.
                             Mixed precision with the paired-bfloat16 or FP32
                             near field, leaf_size <= 64 and stored mode only;
                             elsewhere 2 acts as 1. Its products with several
                             right-hand sides run one vector at a time, and
                             every gather shape runs the bulk-copy kernel.
                             Not in the paper (its library treats the general
                             Y1 x Y2 case, Sec. 6.1). Default 0; other values
                             HM_EINVAL. */
    int on_the_fly;       /* 1: store no factors and no near field: every
                             hm_matvec recomputes the ACA factors of the
                             admissible leaves in passes of consecutive leaves
                             (bounded by scratch_gb) and applies them at once,
                             and evaluates the dense leaves inside the product
                             (the paper's non-precomputed mode, Sec. 5.4).
                             For point sets whose stored H-matrix does not fit
                             the GPU. With symmetric, a pass compresses the
                             canonical leaves of its range and applies them
                             and their mirror leaves (its row sums then depend
                             on the pass count to rounding). With
                             hm_build_batch the passes run over the leaves of
                             all sets in order (a pass may hold leaves of
                             several sets). With rank_model (square matrices)
                             the predicted ranks size the passes. Several
                             right-hand sides run one product each.
                             Default 0. */
    int64_t row_lo, row_hi; /* block-row share of one H-matrix (distributed
                             H-matrices, the outlook of Sec. 7), Morton-order
                             rows [row_lo, row_hi): keep only the leaves whose
                             row cluster meets the range (in symmetric mode
                             also the canonical partners of kept mirror
                             leaves), so that the build compresses and stores
                             only those and the product computes every row of
                             the range exactly as the whole H-matrix does, bit
                             for bit. Rows outside the range then hold
                             incomplete sums: the caller keeps the rows of its
                             range (hm_export_structure's permutation maps
                             Morton rows to points). row_hi <= 0: all rows
                             (default). One point set only (not with
                             hm_build_rect or hm_build_batch). */
} hm_options;

typedef struct hm_handle_s* hm_handle;

/* Fill *opt with the defaults above. */
void hm_options_default(hm_options* opt);

/* Build the H-matrix of A_{phi, Y x Y} (Sec. 5: Morton codes and sort, cluster
 * tree, block cluster tree by level-synchronous traversal (Alg. 1, Alg. 4),
 * batched ACA of the admissible leaves (Alg. 2, Sec. 5.4.1), batched
 * evaluation of the dense leaves (Sec. 5.4.2)).
 *   points    (N, d) row-major doubles, host or device; copied, may be freed
 *             on return
 *   N >= 1, d in {1, 2, 3}, kernel HM_GAUSSIAN | HM_MATERN32 | HM_MATERN_K1
 *   params    [l, sigma^2] (host)
 *   leaf_size C_leaf >= 1; eta >= 0 admissibility parameter
 *   aca_eps   relative Frobenius accuracy of each ACA block; <= 0 selects the
 *             paper's fixed-rank mode with k = k_cap
 * Returns NULL on failure (hm_last_error() says why). */
hm_handle hm_build(const double* points, int64_t N, int d, int kernel,
                   const double* params, int leaf_size, double eta,
                   double aca_eps);

/* As hm_build with options; *status (may be NULL) receives the HM_* code. */
hm_handle hm_build_ex(const double* points, int64_t N, int d, int kernel,
                      const double* params, int leaf_size, double eta,
                      double aca_eps, const hm_options* opt, int* status);

/* Build the H-matrix of A_{phi, Y1 x Y2} for two point sets (Sec. 6.1: the
 * library is for a kernel matrix on sets Y1 and Y2). Each set gets its own
 * Morton order and cluster tree (Sec. 4.4); Alg. 1 runs from the pair of
 * roots, tau a cluster of Y1 and sigma a cluster of Y2; ACA and the dense
 * leaves evaluate phi(y1_i, y2_j).
 *   rows  (N1, d) row-major doubles (Y1), cols (N2, d) (Y2), host or device;
 *         both copied, may be freed on return
 *   params[1] (sigma^2) must be 0: there is no diagonal
 *   the other arguments as hm_build_ex. symmetric and rank_model are
 *   refused (HM_ENOTSUP); on_the_fly is supported. In mixed precision the
 *   global floor of the ACA tests takes the dense leaves' sum of squares as
 *   its lower bound of ||A||_F^2 (a square matrix uses its unit diagonal).
 * hm_matvec / hm_matvec_ex then take x of N2 entries (per vector, in Y2's
 * order) and write y of N1 entries (Y1's order), one product per vector;
 * hm_cg refuses the handle. hm_export_structure writes Y1's permutation
 * followed by Y2's (set-local), leaf pairs (tau in Y1's tree, sigma in Y2's)
 * and hm_export_tree Y1's nodes followed by Y2's.
 * Returns NULL on failure; *status (may be NULL) receives the HM_* code. */
hm_handle hm_build_rect(const double* rows, int64_t N1, const double* cols, int64_t N2, int d,
                        int kernel, const double* params, int leaf_size, double eta,
                        double aca_eps, const hm_options* opt, int* status);

/* y = H x + sigma^2 x (Alg. 3, batched: Sec. 5.4), x and y of length N in the
 * caller's point order, host or device doubles. y is overwritten unless the
 * handle was built with accumulate = 1. */
int hm_matvec(hm_handle h, const double* x, double* y);

/* nrhs right-hand sides stored one after another (x[r*N + i]), results
 * likewise; stream overrides the handle's stream when not NULL.
 * Mixed-precision handles whose leaf slices have at most 64 rows and whose
 * near field is FP64, FP32 or BF16X2 multiply groups of up to 16 vectors in
 * one pass over the stored factors and near field (Alg. 3 applied to the
 * columns of X): a vector's result does not depend on the vectors it is
 * grouped with, and it agrees with the one-vector product to rounding (the
 * two sum in different orders). Other handles run one product per vector.
 * Host x / y are copied per group of 16 vectors. */
int hm_matvec_ex(hm_handle h, const double* x, double* y, int nrhs, void* stream);

/* Release everything the handle owns. NULL-safe. */
void hm_free(hm_handle h);

/* Thread-local description of the last failure ("" if none). */
const char* hm_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far. */
uint64_t hm_kernel_launches(void);

/* Launch shape of the product's gather kernel (Sec. 5.4 batched product; a
 * tuning control, not part of the method). By default (-1) the first product
 * of a kind on a device times every shape once and keeps the fastest for the
 * process. shape 0..4 forces one: 0, 1, 2 = load-based streaming with 8, 16
 * or 4 columns in flight per half-warp (3, 2 or 4 CTAs per SM); 3, 4 =
 * bulk-copy (TMA) pipeline into shared memory with 6 or 4 stages of 64
 * columns (slices of at most 64 rows and formats other than the single
 * bfloat16; otherwise shape 0 runs). A product with the symmetric near
 * field (symmetric = 2) runs the bulk-copy pipeline for every shape: shape 3
 * with 6 stages of 64 columns, shape 2 with 2 stages of 128 columns, the
 * others with 4 stages of 64. Every shape gives bit-identical
 * products. Process-wide, not thread-safe against concurrent products.
 * Returns HM_EINVAL for other values. */
int hm_set_gather_shape(int shape);

/* ACA launch-shape autotuner (Sec. 6.4 tunes the batching parameters by
 * hand; a tuning control, not part of the method). Builds the given problem
 * (arguments as hm_build_ex; on_the_fly must be 0) reps times with each of
 * the shapes 0, 1, 2 of hm_set_aca_shape for every size class, the classes
 * run one after another (profile 2) so that each has its own CUDA-event
 * time, keeps per class the shape of the least time (min over reps), and
 * sets it as by hm_set_aca_shape(class, shape) for later builds. shapes
 * (may be NULL) receives the 12 chosen shapes (-1: class empty, default
 * kept). Shapes give the same approximation up to the order of their sums.
 * On failure the earlier shapes are restored and the build's status is
 * returned. */
int hm_tune_aca_shapes(const double* points, int64_t N, int d, int kernel, const double* params,
                       int leaf_size, double eta, double aca_eps, const hm_options* opt,
                       int reps, int* shapes);

/* Batching sizes (Sec. 5.4.1, bs_ACA; Sec. 5.4.2, bs_dense; a measurement
 * control for the batching study of Sec. 6.4, not part of the method).
 *   aca_entries  > 0: one ACA launch takes consecutive blocks of one size
 *                class and rank bucket while their reserved factor entries
 *                sum_b k_res,b (m_b + n_b) stay <= aca_entries (at least one
 *                block per launch; 1 gives one launch per block);
 *                0 (default): one launch per class and bucket.
 *   gather_items > 0: the one-vector product's gather runs as launches of at
 *                most this many work items (an item is a row tile's U slices and
 *                near-field blocks, up to 4096 columns; 1 gives one launch
 *                per item); 0 (default): one launch.
 * Results do not depend on either: every block and item computes the same
 * values whatever launch it runs in. Process-wide; applies to builds and
 * products started afterwards. Returns HM_EINVAL for negative values. */
int hm_set_batch_limits(int64_t aca_entries, int64_t gather_items);

/* Launch shape of the batched ACA of one block size class (Sec. 5.4.1
 * batching; a tuning control, not part of the method). Size class c holds
 * the admissible blocks with 2^(c+5) < max(m, n) <= 2^(c+6) (class 0 from 1,
 * class 11 unbounded); cls = -1 sets every class. shape -1 (default): the
 * team kernels for classes 0 .. 8 (a team of 1 to 32 warps per block, the
 * residuals in registers, the reductions inside the team), the cluster
 * kernels above; 0: the cluster kernels of the first design for the class
 * (one warp per block up to 512 rows, then a CTA or a thread-block cluster
 * per block); 1: the class's default team shape; 2: another team shape
 * (compiled for float Gaussian builds of classes 2 .. 8; elsewhere the
 * default team shape runs). All compute the
 * same approximation with the same readings of Alg. 2; their sums run in
 * different orders, so results agree to rounding. Blocks whose reservation
 * exceeds 64 ranks always run the cluster kernels. Process-wide; applies to
 * builds started afterwards. Returns HM_EINVAL for other values. */
int hm_set_aca_shape(int cls, int shape);

/* Test hooks of the failure paths (not part of the method; process-wide,
 * applying to builds and products started afterwards; 0 restores the
 * default):
 *   HM_HOOK_ACA_STEP_LIMIT  value > 0 caps the iterations of every block's
 *                           ACA loop at value (default k + n + 1, which no
 *                           block reaches); a block that hits the cap stops
 *                           and the build returns HM_ETIMEOUT.
 *   HM_HOOK_WAIT_LIMIT_NS   value > 0 bounds every mbarrier wait of the
 *                           product's bulk-copy kernels at value ns
 *                           (default 2 s); the producer's final waits for
 *                           copies it issued keep at least 2 s, so no CTA
 *                           exits with a copy into its shared memory in
 *                           flight.
 *   HM_HOOK_GATHER_WITHHOLD value k + 1 > 0: the bulk-copy producer of every
 *                           work item leaves out its chunk k, so that the
 *                           consumers' wait for it runs out; the product
 *                           gives up, sets the status word and returns no
 *                           valid result (see hm_check_status).
 *   HM_HOOK_FAIL_ALLOC      value n > 0: the n-th device allocation of the
 *                           library from now fails as if the device were out
 *                           of memory (HM_ENOMEM); the failing call releases
 *                           what it had allocated.
 *   HM_HOOK_TRAVERSAL_KAPPA value > 0 sets the first level bound of the
 *                           block-tree traversal: level l may hold
 *                           min(4^l, value * 2^l) pairs (default 16, 256 or
 *                           1024 for d = 1, 2, 3, times ceil(1/eta)^d for
 *                           eta < 1). A level that does not fit ends the
 *                           traversal on the device; the host then runs it
 *                           again with the bounds doubled (hm_stats
 *                           traversal_reruns counts these runs).
 *   HM_HOOK_TRAVERSAL_TRIES value n > 0: at most n traversals (default 16);
 *                           if the n-th still does not fit the build
 *                           returns HM_EOVERFLOW.
 * Returns HM_EINVAL for an unknown hook or a value out of range. */
enum {
    HM_HOOK_ACA_STEP_LIMIT = 0,
    HM_HOOK_WAIT_LIMIT_NS = 1,
    HM_HOOK_GATHER_WITHHOLD = 2,
    HM_HOOK_FAIL_ALLOC = 3,
    HM_HOOK_TRAVERSAL_KAPPA = 4,
    HM_HOOK_TRAVERSAL_TRIES = 5
};
int hm_set_test_hook(int hook, int64_t value);

/* Device status of a handle's earlier calls: synchronises the handle's
 * stream and returns HM_ETIMEOUT if a bounded device loop or wait gave up
 * since the last check (the status word is then cleared), else HM_OK. A
 * product whose y is in host memory does this check itself before it
 * returns; a product on device buffers (and one captured in a CUDA graph)
 * leaves it to this call. */
int hm_check_status(hm_handle h);

/* Device bytes the library holds at this moment, over every handle, batch
 * and call in flight (the allocations it made and has not yet released; the
 * fixed array of the allocation-free sort is not counted). For checks that a
 * failed call released what it had allocated. */
uint64_t hm_device_bytes(void);

/* Counts, ranks and bytes of a built handle. */
typedef struct hm_stats {
    int64_t n_points, n_nodes, n_adm, n_dense, n_tiles;
    int depth, d;
    int64_t sum_rank;           /* sum of ACA ranks */
    int max_rank;
    int64_t rank_cap_hits;      /* blocks that stopped at the rank cap */
    int64_t n_rejected;         /* rejected ACA columns, all blocks */
    int64_t n_mispredicted;     /* rank model: blocks re-run with k_cap */
    int64_t factor_entries;     /* sum_b k_b (m_b + n_b) */
    int64_t near_entries;       /* sum over dense leaves m_b n_b */
    int64_t factor_bytes, near_bytes;
    int64_t mvp_bytes;          /* algorithmic bytes moved by one product */
    int64_t reserved_factor_entries; /* storage reserved for the factors */
    double t_structure_ms, t_aca_ms, t_dense_ms, t_total_ms; /* last build */
    int aca_passes;             /* scratch passes of the plain ACA */
    int precision, near_format;
    int64_t aca_evals;          /* kernel evaluations done by ACA */
    double aca_flops;           /* algorithmic ACA flops: evals * flops per
                                   evaluation + sum_b 2 k_b (k_b - 1)(m_b + n_b) */
    /* profile = 1: sums over the products since the last hm_get_stats */
    int64_t mvp_count;
    double t_mvp_ms, t_mvp_gather_ms, t_mvp_vtx_ms, t_mvp_tile_ms;
    int64_t mvp_vtx_bytes, mvp_tile_bytes;  /* algorithmic bytes per product of
                                               V^T x and of the main gather kernel */
    /* last build: ACA time per block size class (class c: 2^(c+5) < max(m, n)
       <= 2^(c+6); class 0 from 1, class 11 unbounded), CUDA events on each
       class's stream (the classes run concurrently), summed over passes */
    double t_aca_class_ms[12];
    /* profile = 1 on an on-the-fly handle: sums over the products since the
       last hm_get_stats of the time in the ACA passes, in the low-rank apply
       (t = V^T x and U t of each pass) and in the dense leaves; aca_evals and
       aca_flops then count the ACA work of one product, near_entries the
       dense entries evaluated per product */
    double t_np_aca_ms, t_np_lowrank_ms, t_np_near_ms;
    /* last build: traversals run again because a level of the block tree
       did not fit its bound (summed over the point sets) */
    int traversal_reruns;
    /* profile = 1: the product's time and algorithmic bytes after its main
       gather kernel (t_mvp_tile_ms, mvp_tile_bytes): the finish that writes
       y and, with symmetric = 2, the mirror blocks' t and the gather of the
       mirror slices (sums over the products since the last hm_get_stats) */
    double t_mvp_tail_ms;
    int64_t mvp_tail_bytes;
} hm_stats;

int hm_get_stats(hm_handle h, hm_stats* out);

/* Structure for parity checks (all host arrays, caller-allocated):
 *   codes[N] (uint64, input order), perm[N] (int64: Morton position ->
 *   input index), adm[2*n_adm] and dense[2*n_dense] (int64 node-id pairs in
 *   canonical (tau.lo, sigma.lo) order), ranks[n_adm] (int32). Any may be NULL. */
int hm_export_structure(hm_handle h, uint64_t* codes, int64_t* perm,
                        int64_t* adm, int64_t* dense, int32_t* ranks);

/* Cluster-tree node ranges and bounding boxes (host arrays of n_nodes and
 * n_nodes*d entries; absent nodes have lo = hi = -1). */
int hm_export_tree(hm_handle h, int64_t* lo, int64_t* hi, double* bbmin,
                   double* bbmax);

/* Factors of admissible leaf b (canonical index): U (m, k) and V (n, k)
 * column-major doubles into host arrays of m*k_cap and n*k_cap entries;
 * *rank receives k. Converted to double in mixed precision. */
int hm_export_factors(hm_handle h, int64_t b, double* U, double* V, int* rank);

/* Conjugate gradients on (H + sigma^2 I) x = b (Sec. 1, with the H-MVP as
 * the operator): FP64 inner products and vector updates on the device. x
 * holds the start vector on entry (host or device). Stops when
 * ||r_k|| / ||b|| <= rtol or after maxit iterations. */
int hm_cg(hm_handle h, const double* b, double* x, double rtol, int maxit,
          int* iters, double* relres);

/* ------------------------------------------------------------------------
 * Batched form: many independent point sets built and multiplied together
 * (Sec. 4.2 batching applied across problems). points_all holds the sets one
 * after another ((sum N_s), d_s per set, row-major), x_all / y_all likewise.
 * All sets share one plan: their blocks go through the same size-class ACA
 * launches and one gather per product. opt as hm_build_ex; on_the_fly runs
 * the passes over the leaves of all sets in order (a pass may hold leaves
 * of several sets); a block-row share (row_lo, row_hi) is refused
 * (HM_ENOTSUP).
 * ------------------------------------------------------------------------ */
typedef struct hm_batch_s* hm_batch;

hm_batch hm_build_batch(int nsets, const double* points_all, const int64_t* N,
                        const int* d, int kernel, const double* params,
                        int leaf_size, double eta, double aca_eps,
                        const hm_options* opt, int* status);
int hm_matvec_batch(hm_batch b, const double* x_all, double* y_all);
int hm_batch_stats(hm_batch b, hm_stats* out);
void hm_free_batch(hm_batch b);

/* ------------------------------------------------------------------------
 * Learned rank model (not in the paper): MLP 8 -> 64 -> 64 -> 1 with ReLU,
 * FP32. theta = [W1 (64x8 row-major), b1 (64), W2 (64x64), b2 (64),
 * W3 (1x64), b3 (1)] = 4801 floats. Features per admissible block:
 *   f = [d/3, log2|tau|/16, log2|sigma|/16, log2(1+diam_tau/l),
 *        log2(1+diam_sigma/l), log2(1+dist/l), -log10(eps)/8, kernel]
 * and the target is log2(1 + ACA rank).
 * ------------------------------------------------------------------------ */
#define HM_MLP_NPARAM 4801

/* Features (n_adm x 8 floats) and ranks of a built handle (device or host). */
int hm_block_features(hm_handle h, float* feats, float* target);

/* out[n] = MLP(F[n x 8]) (device or host pointers). */
int hm_mlp_forward(const float* theta, const float* F, int64_t n, float* out,
                   void* stream);

/* Mean squared error of MLP(F) against target and its gradient grad[4801]
 * (device pointers). *loss may be NULL. */
int hm_mlp_loss_grad(const float* theta, const float* F, const float* target,
                     int64_t n, float* grad, float* loss, void* stream);

/* One Adam step (device pointers), step count t >= 1. */
int hm_mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t t,
                float lr, float b1, float b2, float eps, void* stream);

/* ------------------------------------------------------------------------
 * Device helpers exposed for parity tests of the individual build steps.
 * ------------------------------------------------------------------------ */

/* Morton codes of N points (device in/out). bits per dimension is
 * min(32, 64/d); the box is the points' global min/max. */
int hm_morton_codes(const double* points, int64_t N, int d, uint64_t* codes,
                    void* stream);

/* Stable LSD radix sort of (key, value) pairs on the device, in place,
 * sorting on the low key_bits bits of the keys. */
int hm_radix_sort_pairs(uint64_t* keys, uint32_t* values, int64_t n,
                        int key_bits, void* stream);

/* ------------------------------------------------------------------------
 * Allocation-free sort. The paper has no counterpart: this entry point is
 * for callers that cannot allocate device memory while they run, such as a
 * program that has handed all free device memory to its own pool or caching
 * allocator, or a latency-critical loop that must not block on an
 * allocation. It sorts like hm_radix_sort_pairs (stable LSD radix sort of
 * (key, value) pairs on the low key_bits bits, in place) but allocates
 * nothing: no cudaMalloc, cudaFree or allocating library call.
 *   keys, values  device pointers, n entries each (sorted in place)
 *   n             at most HM_NOALLOC_SORT_MAX; larger n returns HM_EINVAL
 *                 and leaves the arrays untouched
 * Its scratch is one fixed array of about 3.3 MB in the library's device
 * memory, held by every GPU that loads the library until the process ends.
 * The first call on each device looks up that array's address (with that
 * device current); make that first call before any stream capture. All calls
 * on a device share the array, so calls that overlap on the GPU (on streams
 * without an order between them) race and give wrong results. */
#define HM_NOALLOC_SORT_MAX 262144
int hm_radix_sort_pairs_noalloc(uint64_t* keys, uint32_t* values, int64_t n, int key_bits,
                                void* stream);

/* ------------------------------------------------------------------------
 * Measured arithmetic peak. Not part of the paper's method: it gives the
 * denominator of the roofline fractions of the ALU-bound kernels (ACA, dense
 * evaluation). A kernel of independent fused multiply-add chains fills every
 * SM of the current device; the best of three launches, timed with CUDA
 * events, gives *flops in FLOP/s (one FMA counts 2).
 *   precision  HM_PREC_MIXED: FP32 FMA;  HM_PREC_FP64: FP64 FMA
 *   flops      host pointer, written on success
 * Synchronises the device. Returns HM_EINVAL for a NULL pointer or an unknown
 * precision, HM_ECUDA if a CUDA call fails. */
int hm_alu_peak(int precision, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* HM_H */
