/*
 * hm_oracle.h -- CPU oracle of the H-matrix build and H-matrix-vector product
 * of P. Zaspel, "Algorithmic patterns for H-matrices on many-core processors"
 * (arXiv 1708.09707).
 *
 * TEST INFRASTRUCTURE. Plain, slow, single-threaded C in double precision,
 * compiled without floating-point contraction. Only the test suite, the
 * package's smoke check and the benchmark's CPU-baseline leg load it. It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Pins (the tests that tie each function to something other than itself):
 *   or_morton        hand-derived codes (tests/golden/morton_codes.txt) and the
 *                    recursive quadrant/octant order of grid points
 *   or_sort          numpy's stable argsort
 *   or_tree_ranges   closed form of the halving rule (sizes, leaf count)
 *   or_bbox          numpy min/max per range
 *   or_admissible    hand-placed boxes with known diam/dist (golden file)
 *   or_build leaves  tiling of I x I (brute-force coverage bitmap) and the
 *                    Alg. 1 invariants; a hand-derived 1-D leaf list
 *   or_aca           exact rank-r matrices, cross-interpolation property,
 *                    Eckart-Young lower bound from numpy's SVD
 *   or_matvec        eta = 0 and C >= N reduce to the dense product; error
 *                    against brute force within O(eps); symmetry; sigma^2 x
 *   or_dense_matvec  numpy dense matrix product
 *   or_build_rect    Y2 = Y1 gives the square build bit for bit; leaves tile
 *                    I1 x I2 once; eta = 0 and C >= max(N1, N2) reduce to
 *                    the dense product; error against or_dense_matvec_rect
 *                    within O(eps); A(Y1,Y2) and A(Y2,Y1) are transposes
 *   or_dense_matvec_rect  numpy dense matrix product
 *   or_cg            numpy.linalg.solve on the same dense system
 *   or_mlp_*         central finite differences; closed-form first Adam step
 */
#ifndef HM_ORACLE_H
#define HM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Kernel ids: 0 = Gaussian exp(-r^2/l^2), 1 = Matern-3/2 (1+sqrt3 r/l)e^{-sqrt3 r/l},
 * 2 = Matern of order 1, (r/l) K_1(r/l) (phi(0) = 1). */
double or_kernel_eval(int kernel, double ell, const double* a, const double* b, int d);

/* Sec. 4.4, Alg. 6: Morton codes. pts row-major (N,d). Writes codes[N] and the
 * global box lo[d], hi[d] and per-dimension scale[d]. Returns bits per dim. */
int or_morton(const double* pts, int64_t N, int d, uint64_t* codes,
              double* lo, double* hi, double* scale);

/* Stable sort of point indices by Morton code (Sec. 4.4). perm[j] = original
 * index of the j-th point in Morton order. */
void or_sort(const uint64_t* codes, int64_t N, int64_t* perm);

/* Cluster tree of Sec. 2.1 with cardinality-based halving (Sec. 4.4): node
 * ids in heap order, absent nodes get lo = hi = -1. */
int or_tree_depth(int64_t N, int C);
int64_t or_tree_nodes(int64_t N, int C);
void or_tree_ranges(int64_t N, int C, int64_t* lo, int64_t* hi);

/* Bounding boxes Q_tau (Sec. 2.2) of every present node; coords_m is the
 * Morton-ordered point array, row-major (N,d). bbmin/bbmax are (nodes, d). */
void or_bbox(const double* coords_m, int64_t N, int d, int C,
             const int64_t* lo, const int64_t* hi, double* bbmin, double* bbmax);

/* Eq. (admissibilityCondition) in squared form. use_max selects max{diam}. */
int or_admissible(const double* amin, const double* amax, const double* bmin,
                  const double* bmax, int d, double eta2, int use_max);

/* Entry callback for ACA on an explicit matrix (tests). */
typedef double (*or_entry_fn)(const void* ctx, int64_t i, int64_t j);

/* Alg. 2 (ACA) with the readings stated in hm_oracle.c. U is (m, k_cap) and V
 * is (n, k_cap), column-major: column l of U starts at U + l*m. Returns the
 * rank; piv_i/piv_j (k_cap each, may be NULL) receive the pivots, n_rej the
 * number of rejected columns. */
int or_aca(or_entry_fn f, const void* ctx, int64_t m, int64_t n, double eps,
           int k_cap, double aca_eta, double eps0, double* U, double* V,
           int64_t* piv_i, int64_t* piv_j, int64_t* n_rej);

/* ACA on a dense column-major (m,n) matrix: A[i + j*m]. */
int or_aca_dense(const double* A, int64_t m, int64_t n, double eps, int k_cap,
                 double aca_eta, double eps0, double* U, double* V,
                 int64_t* piv_i, int64_t* piv_j, int64_t* n_rej);

typedef struct or_hmat or_hmat;

/* The whole build: Morton, sort, cluster tree, boxes, Alg. 1, ACA of every
 * admissible leaf. params[0] = l, params[1] = sigma^2. aca_eps <= 0 selects
 * the paper's fixed-rank mode with k = k_cap. eps0 <= 0 selects 1e-14. */
or_hmat* or_build(const double* pts, int64_t N, int d, int kernel,
                  const double* params, int C, double eta, int adm_max,
                  double aca_eps, int k_cap, double aca_eta, double eps0);
void or_free(or_hmat* h);

/* A_{phi, Y1 x Y2} for two point sets (Sec. 6.1: the paper's library builds
 * A for sets Y1 and Y2): each set is ordered and clustered on its own, Alg. 1
 * runs from the pair of roots with tau in Y1's tree and sigma in Y2's, ACA
 * entries are phi(y1_i, y2_j). params[1] (sigma^2) is ignored: there is no
 * diagonal. The product maps x of length N2 to y of length N1. */
or_hmat* or_build_rect(const double* pts1, int64_t N1, const double* pts2, int64_t N2,
                       int d, int kernel, const double* params, int C, double eta,
                       int adm_max, double aca_eps, int k_cap, double aca_eta, double eps0);
or_hmat* or_build_structure_rect(const double* pts1, int64_t N1, const double* pts2,
                                 int64_t N2, int d, int kernel, const double* params, int C,
                                 double eta, int adm_max);
/* Column side (Y2) of a rectangular handle; the row side for a square one. */
int64_t or_n_cols(const or_hmat* h);
int64_t or_n_nodes_cols(const or_hmat* h);
void or_get_col_perm(const or_hmat* h, int64_t* perm);
void or_get_col_tree(const or_hmat* h, int64_t* lo, int64_t* hi, double* bbmin, double* bbmax);

/* Structure only (no ACA): for the large-N parity of integer structure. */
or_hmat* or_build_structure(const double* pts, int64_t N, int d, int kernel,
                            const double* params, int C, double eta, int adm_max);

/* Symmetric kernels: every admissible leaf (sigma, tau) with lo[sigma] >
 * lo[tau] takes the factors of (tau, sigma) with U and V exchanged (call
 * after compression of all leaves). */
void or_mirror_transposed(or_hmat* h);

/* ACA of admissible leaves [b0, b1) only (builds the factors of those). */
/* Threads of the block loops of ACA and the product (1: plain loops). */
void or_set_threads(int t);
/* ACA of the listed admissible leaves (factors stored in list order). */
void or_compress_ids(or_hmat* h, const int64_t* ids, int64_t n_ids, double aca_eps,
                     int k_cap, double aca_eta, double eps0);
void or_compress_range(or_hmat* h, int64_t b0, int64_t b1, double aca_eps,
                       int k_cap, double aca_eta, double eps0);

/* Sizes and exports. */
int64_t or_n_adm(const or_hmat* h);
int64_t or_n_dense(const or_hmat* h);
int64_t or_n_nodes(const or_hmat* h);
void or_get_codes(const or_hmat* h, uint64_t* codes);
void or_get_perm(const or_hmat* h, int64_t* perm);
void or_get_coords(const or_hmat* h, double* coords_m);
void or_get_tree(const or_hmat* h, int64_t* lo, int64_t* hi, double* bbmin, double* bbmax);
/* leaves: (n, 2) node ids (tau, sigma) in canonical (tau.lo, sigma.lo) order. */
void or_get_adm(const or_hmat* h, int64_t* leaves);
void or_get_dense(const or_hmat* h, int64_t* leaves);
void or_get_ranks(const or_hmat* h, int32_t* ranks, int64_t* n_rej);
/* Factors of adm leaf b: U (m, rank) and V (n, rank), column-major. */
void or_get_factors(const or_hmat* h, int64_t b, double* U, double* V);
void or_get_pivots(const or_hmat* h, int64_t b, int64_t* piv_i, int64_t* piv_j);

/* Alg. 3: y = H x (+ sigma^2 x), x and y in the caller's point order. */
void or_matvec(const or_hmat* h, const double* x, double* y);
/* Rows [r0, r1) of the Morton-ordered product from the Morton-ordered x_m,
 * from the leaves that touch them (block-row share; bit for bit or_matvec's
 * rows). */
void or_matvec_rows(const or_hmat* h, const double* xm, int64_t r0, int64_t r1, double* yr);

/* Brute force y_i = sum_j phi(y_i, y_j) x_j + sigma^2 x_i (Neumaier sums). */
void or_dense_matvec(const double* pts, int64_t N, int d, int kernel,
                     const double* params, const double* x, double* y);
/* Brute force of A_{phi, Y1 x Y2} x (Neumaier sums over the N2 columns). */
void or_dense_matvec_rect(const double* pts1, int64_t N1, const double* pts2, int64_t N2,
                          int d, int kernel, const double* params, const double* x,
                          double* y);
/* The same for a subset of rows: y_rows[r] for row index rows[r]. */
void or_dense_rows(const double* pts, int64_t N, int d, int kernel,
                   const double* params, const int64_t* rows, int64_t nrows,
                   const double* x, double* y_rows);

/* Conjugate gradients on (A_H + sigma^2 I) x = b (Sec. 1). x holds the start
 * vector on entry. Returns iterations; relres = ||r_k|| / ||b||. */
int or_cg(const or_hmat* h, const double* b, double* x, double rtol, int maxit,
          double* relres);

/* Rank-model features of the admissible leaves (n_adm, 8). */
void or_block_features(const or_hmat* h, double aca_eps, double* feats);

/* MLP 8 -> 64 -> 64 -> 1 (ReLU). theta = [W1 (64x8), b1, W2 (64x64), b2,
 * W3 (1x64), b3], 4801 values. */
#define OR_MLP_NPARAM 4801
void or_mlp_forward(const double* theta, const double* F, int64_t n, double* out);
/* Mean-squared error and its gradient (grad may be NULL). */
double or_mlp_loss_grad(const double* theta, const double* F, const double* target,
                        int64_t n, double* grad);
/* One Adam step at step count t (1-based). */
void or_adam_step(double* theta, const double* grad, double* m, double* v,
                  int64_t n, int64_t t, double lr, double b1, double b2, double eps);

#ifdef __cplusplus
}
#endif
#endif
