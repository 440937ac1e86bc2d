/*
 * hm_oracle.c -- CPU oracle of the H-matrix build and H-MVP of P. Zaspel,
 * "Algorithmic patterns for H-matrices on many-core processors" (arXiv
 * 1708.09707).
 *
 * TEST INFRASTRUCTURE ONLY (see hm_oracle.h for the pins). Single-threaded,
 * double precision, compiled with -O2 -ffp-contract=off so that no multiply
 * and add are fused. Everything here follows the paper's definitions and
 * algorithms in the paper's order; where the paper is silent the reading used
 * is stated beside the code.
 */
#include "hm_oracle.h"

#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Kernel functions (Sec. 6.2 model problem; the length scale l and the     */
/* Matern order 3/2 are the workloads' parameters).                          */
/*   Gaussian:    phi = exp(-(D2 * (1/(l*l))))                               */
/*   Matern-3/2:  s = sqrt(D2) * (sqrt(3)/l),  phi = (1 + s) * exp(-s)       */
/*   Matern K_1:  s = sqrt(D2) / l,  phi = s * K_1(s), phi(0) = 1: Sec. 6.2's */
/*                Matern kernel with beta - d/2 = 1 without its constant      */
/*                factor 1/(2^(beta-1) Gamma(beta)) (reading: a constant      */
/*                factor of the whole matrix changes no block, rank or        */
/*                relative error).                                            */
/* D2 = sum_i (a_i - b_i)^2 accumulated over i = 0..d-1.                     */
/* ------------------------------------------------------------------------ */

/* K_1(x), x > 0, the modified Bessel function of the second kind of order 1.
 * x <= 2: the ascending series (Abramowitz and Stegun 9.6.11 with n = 1)
 *   K_1(x) = 1/x + ln(x/2) I_1(x)
 *            - (x/4) sum_k (psi(k+1) + psi(k+2)) (x^2/4)^k / (k! (k+1)!),
 *   I_1(x) = (x/2) sum_k (x^2/4)^k / (k! (k+1)!), psi(k+1) = -gamma + H_k,
 *   summed over 20 terms (the 20th is below 1e-37 of the first).
 * x > 2: the integral K_1(x) = int_0^inf exp(-x cosh u) cosh u du (A&S
 *   9.6.24) by the trapezoidal rule with the step h = 0.2 / sqrt(x), up to
 *   where x (cosh u - 1) exceeds 60 (the integrand is then below e^-60 of
 *   its value at 0). The integrand is entire, so the rule's relative error is
 *   about exp(x (1 - cos a) - 2 pi a / h) for a strip half-width a < pi/2:
 *   below e^-60 with a = min(1.5, 10 / sqrt(x)), far below rounding. */
static double or_bessel_k1(double x)
{
    if (x <= 2.0) {
        const double euler_gamma = 0.57721566490153286061;
        double q = 0.25 * x * x;
        double term = 1.0;                 /* (x^2/4)^k / (k! (k+1)!) */
        double Hk = 0.0;                   /* H_k */
        double sum_i = 0.0, sum_psi = 0.0;
        for (int k = 0; k < 20; ++k) {
            double Hk1 = Hk + 1.0 / (double)(k + 1);
            double psi_sum = (-euler_gamma + Hk) + (-euler_gamma + Hk1);
            sum_i = sum_i + term;
            sum_psi = sum_psi + psi_sum * term;
            term = term * q / ((double)(k + 1) * (double)(k + 2));
            Hk = Hk1;
        }
        double I1 = 0.5 * x * sum_i;
        return 1.0 / x + log(0.5 * x) * I1 - 0.25 * x * sum_psi;
    } else {
        double h = 0.2 / sqrt(x);
        double sum = 0.5 * exp(-x);        /* half weight at u = 0 */
        for (int64_t j = 1;; ++j) {
            double u = (double)j * h;
            double sh = sinh(0.5 * u);
            double cm1 = 2.0 * sh * sh;    /* cosh(u) - 1 without cancellation */
            if (x * cm1 > 60.0) break;
            sum = sum + exp(-x * (1.0 + cm1)) * (1.0 + cm1);
        }
        return h * sum;
    }
}

double or_kernel_eval(int kernel, double ell, const double* a, const double* b, int d)
{
    double D2 = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = a[i] - b[i];
        D2 = D2 + t * t;
    }
    if (kernel == 0) {
        double c = 1.0 / (ell * ell);
        return exp(-(D2 * c));
    } else if (kernel == 1) {
        double c = sqrt(3.0) / ell;
        double s = sqrt(D2) * c;
        return (1.0 + s) * exp(-s);
    } else {
        if (D2 == 0.0) return 1.0;         /* lim_{s -> 0} s K_1(s) = 1 */
        double s = sqrt(D2) / ell;
        return s * or_bessel_k1(s);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.4, Alg. 6: Morton codes.                                           */
/* Readings (the paper leaves these open): b = min(32, floor(64/d)) bits per */
/* dimension; the normalisation box is the global min/max of the points;     */
/* fixed point q_i = min(floor((x_i - lo_i) * s_i), 2^b - 1) with            */
/* s_i = 2^b / (hi_i - lo_i) (0 if hi_i == lo_i); bit t of q_i goes to code  */
/* bit t*d + (d-1-i), so dimension 0 is the most significant in each group. */
/* The stretch and interleave are done one bit at a time.                    */
/* ------------------------------------------------------------------------ */
int or_morton(const double* pts, int64_t N, int d, uint64_t* codes,
              double* lo, double* hi, double* scale)
{
    int b = 64 / d;
    if (b > 32) b = 32;
    for (int i = 0; i < d; ++i) {
        lo[i] = pts[i];
        hi[i] = pts[i];
    }
    for (int64_t p = 1; p < N; ++p)
        for (int i = 0; i < d; ++i) {
            double x = pts[p * d + i];
            if (x < lo[i]) lo[i] = x;
            if (x > hi[i]) hi[i] = x;
        }
    double full = ldexp(1.0, b);
    uint64_t qmax = (b == 64) ? ~0ull : ((1ull << b) - 1ull);
    for (int i = 0; i < d; ++i)
        scale[i] = (hi[i] > lo[i]) ? full / (hi[i] - lo[i]) : 0.0;
    for (int64_t p = 0; p < N; ++p) {
        uint64_t code = 0;
        for (int i = 0; i < d; ++i) {
            double f = floor((pts[p * d + i] - lo[i]) * scale[i]);
            uint64_t q = (f >= (double)qmax) ? qmax : (uint64_t)f;
            for (int t = 0; t < b; ++t) {
                uint64_t bit = (q >> t) & 1ull;
                code |= bit << (t * d + (d - 1 - i));
            }
        }
        codes[p] = code;
    }
    return b;
}

/* ------------------------------------------------------------------------ */
/* Stable sort by Morton code (Sec. 4.4 sorts the points by their codes;    */
/* ties keep the input order, i.e. a stable sort).                           */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t code; int64_t idx; } or_pair;

static int or_pair_cmp(const void* a, const void* b)
{
    const or_pair* x = (const or_pair*)a;
    const or_pair* y = (const or_pair*)b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

void or_sort(const uint64_t* codes, int64_t N, int64_t* perm)
{
    or_pair* p = (or_pair*)malloc((size_t)N * sizeof(or_pair));
    for (int64_t i = 0; i < N; ++i) {
        p[i].code = codes[i];
        p[i].idx = i;
    }
    qsort(p, (size_t)N, sizeof(or_pair), or_pair_cmp);
    for (int64_t i = 0; i < N; ++i) perm[i] = p[i].idx;
    free(p);
}

/* ------------------------------------------------------------------------ */
/* Cluster tree (Sec. 2.1, conditions C1-C4) by cardinality-based halving    */
/* of the Morton-ordered index range (Sec. 4.4): node [lo,hi) splits iff     */
/* hi - lo > C, into [lo, lo+(hi-lo)/2) and [lo+(hi-lo)/2, hi) (the left     */
/* child takes the floor). Heap numbering: root 0, children 2v+1, 2v+2.      */
/* ------------------------------------------------------------------------ */
int or_tree_depth(int64_t N, int C)
{
    int depth = 0;
    int64_t s = N; /* largest node size on the current level */
    while (s > C) {
        s = s - s / 2;
        depth++;
    }
    return depth;
}

int64_t or_tree_nodes(int64_t N, int C)
{
    return (2ll << or_tree_depth(N, C)) - 1;
}

static void or_tree_fill(int64_t v, int64_t lo, int64_t hi, int C,
                         int64_t* L, int64_t* H)
{
    L[v] = lo;
    H[v] = hi;
    if (hi - lo > C) {
        int64_t mid = lo + (hi - lo) / 2;
        or_tree_fill(2 * v + 1, lo, mid, C, L, H);
        or_tree_fill(2 * v + 2, mid, hi, C, L, H);
    }
}

void or_tree_ranges(int64_t N, int C, int64_t* lo, int64_t* hi)
{
    int64_t n = or_tree_nodes(N, C);
    for (int64_t v = 0; v < n; ++v) {
        lo[v] = -1;
        hi[v] = -1;
    }
    or_tree_fill(0, 0, N, C, lo, hi);
}

/* Sec. 2.2: Q_tau = prod_i [min_{j in tau} y_j^(i), max_{j in tau} y_j^(i)]. */
void or_bbox(const double* coords_m, int64_t N, int d, int C,
             const int64_t* lo, const int64_t* hi, double* bbmin, double* bbmax)
{
    int64_t n = or_tree_nodes(N, C);
    for (int64_t v = 0; v < n; ++v) {
        for (int i = 0; i < d; ++i) {
            bbmin[v * d + i] = 0.0;
            bbmax[v * d + i] = 0.0;
        }
        if (lo[v] < 0) continue;
        for (int i = 0; i < d; ++i) {
            double a = coords_m[lo[v] * d + i], b = a;
            for (int64_t j = lo[v] + 1; j < hi[v]; ++j) {
                double x = coords_m[j * d + i];
                if (x < a) a = x;
                if (x > b) b = x;
            }
            bbmin[v * d + i] = a;
            bbmax[v * d + i] = b;
        }
    }
}

/* Eq. (admissibilityCondition), squared: min{D2_tau, D2_sigma} <= eta^2 G2  */
/* with D2 = sum_i (b_i - a_i)^2 and G2 = sum_i (g1^2 + g2^2),               */
/* g1 = max(0, a_tau - b_sigma), g2 = max(0, a_sigma - b_tau). The sums run  */
/* over i = 0..d-1 in that order; eta2 = eta*eta is formed once.            */
int or_admissible(const double* amin, const double* amax, const double* bmin,
                  const double* bmax, int d, double eta2, int use_max)
{
    double Dt = 0.0, Ds = 0.0, G2 = 0.0;
    for (int i = 0; i < d; ++i) {
        double et = amax[i] - amin[i];
        double es = bmax[i] - bmin[i];
        Dt = Dt + et * et;
        Ds = Ds + es * es;
        double g1 = amin[i] - bmax[i];
        double g2 = bmin[i] - amax[i];
        if (g1 < 0.0) g1 = 0.0;
        if (g2 < 0.0) g2 = 0.0;
        G2 = G2 + (g1 * g1 + g2 * g2);
    }
    double D = use_max ? (Dt > Ds ? Dt : Ds) : (Dt < Ds ? Dt : Ds);
    return D <= eta2 * G2;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: ACA with partial pivoting.                                        */
/* Readings of the paper (Sec. 2.4 leaves them open):                        */
/*  - first column j_1 = 0; later columns: argmax over unused columns of the */
/*    residual of a reference row, lowest index on ties. The reference row  */
/*    starts at row 0; once its residual is resolved (max <= tol times the   */
/*    RMS row norm sqrt(S2/m) of the approximation, tol = eps, or eps0 in    */
/*    fixed-rank mode) it moves to the lowest row not yet used as pivot or   */
/*    reference (at most once per step).                                     */
/*    The residual row v_r of the pivot row is not used for the choice: next */
/*    to the current column j_r it is nearly maximal at the columns of close */
/*    or duplicate points, which adds nearly redundant crosses;              */
/*  - row pivot i_r = argmax |u^_r| (lowest index on ties);                  */
/*  - the paper asks for a column with ||u^|| > eps0, eps0 near machine     */
/*    precision, and leaves the search open: a column whose largest residual */
/*    entry is <= eps0 * max_i |A(i,j)| is rejected, the lowest unused       */
/*    column is tried next and r does not advance; after OR_REJ_RUN          */
/*    rejections in a row the block is taken as fully approximated (the      */
/*    search is bounded instead of scanning every column);                   */
/*  - the eta in the stopping rule is a separate aca_eta (the admissibility  */
/*    eta = 1 of the workloads would make the rule never fire);              */
/*  - ||sum_l u_l v_l^T||_F^2 is updated by the textbook recursion           */
/*    S2 += 2 sum_{l<r} (u_r.u_l)(v_l.v_r) + |u_r|^2 |v_r|^2;                */
/*  - stop when |u_r| |v_r| <= eps (1-aca_eta)/(1+eps) sqrt(S2) (eps relative */
/*    to the approximation's own norm) and the reference row is resolved;    */
/*    eps <= 0 is the paper's fixed-rank mode (no test, k = k_cap);          */
/*  - the rank never exceeds min(k_cap, m, n).                               */
/* ------------------------------------------------------------------------ */
#define OR_REJ_RUN 4

int or_aca(or_entry_fn f, const void* ctx, int64_t m, int64_t n, double eps,
           int k_cap, double aca_eta, double eps0, double* U, double* V,
           int64_t* piv_i, int64_t* piv_j, int64_t* n_rej)
{
    int64_t kmax = k_cap;
    if (kmax > m) kmax = m;
    if (kmax > n) kmax = n;
    if (eps0 <= 0.0) eps0 = 1e-14;
    unsigned char* used = (unsigned char*)calloc((size_t)n, 1);
    unsigned char* seen = (unsigned char*)calloc((size_t)m, 1); /* pivot/reference rows */
    double* uh = (double*)malloc((size_t)m * sizeof(double));
    double* rr = (double*)malloc((size_t)n * sizeof(double));   /* reference row residual */
    double thr = (eps > 0.0) ? eps * (1.0 - aca_eta) / (1.0 + eps) : -1.0;
    double rtol = (eps > 0.0) ? eps : eps0;
    double S2 = 0.0;
    int r = 0;
    int64_t j = 0, rej = 0, run = 0;
    int64_t iref = 0;
    seen[0] = 1;
    for (int64_t c = 0; c < n; ++c) rr[c] = f(ctx, 0, c);

    while (r < kmax) {
        /* residual column u^_r = A(:, j) - sum_{l<r} u_l (v_l)_j */
        used[j] = 1;
        double amax = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            double a = f(ctx, i, j);
            if (fabs(a) > amax) amax = fabs(a);
            double s = a;
            for (int l = 0; l < r; ++l) s = s - U[l * m + i] * V[l * n + j];
            uh[i] = s;
        }
        /* row pivot: |u^_{i_r}| = ||u^||_inf */
        int64_t is = 0;
        double best = fabs(uh[0]);
        for (int64_t i = 1; i < m; ++i)
            if (fabs(uh[i]) > best) {
                best = fabs(uh[i]);
                is = i;
            }
        if (!(best > eps0 * amax)) {
            /* column already represented: try the lowest unused one */
            rej++;
            if (++run >= OR_REJ_RUN) break;
            int64_t jn = -1;
            for (int64_t c = 0; c < n; ++c)
                if (!used[c]) {
                    jn = c;
                    break;
                }
            if (jn < 0) break;
            j = jn;
            continue;
        }
        run = 0;
        /* u_r = u^_r / u^_{i_r} */
        double piv = uh[is];
        double* u = U + (int64_t)r * m;
        for (int64_t i = 0; i < m; ++i) u[i] = uh[i] / piv;
        /* v_r = A(i_r, :)^T - sum_{l<r} (u_l)_{i_r} v_l */
        double* v = V + (int64_t)r * n;
        for (int64_t c = 0; c < n; ++c) {
            double s = f(ctx, is, c);
            for (int l = 0; l < r; ++l) s = s - U[l * m + is] * V[l * n + c];
            v[c] = s;
        }
        if (piv_i) piv_i[r] = is;
        if (piv_j) piv_j[r] = j;
        /* Frobenius norm of the approximation, updated */
        double nu2 = 0.0, nv2 = 0.0, cross = 0.0;
        for (int64_t i = 0; i < m; ++i) nu2 = nu2 + u[i] * u[i];
        for (int64_t c = 0; c < n; ++c) nv2 = nv2 + v[c] * v[c];
        for (int l = 0; l < r; ++l) {
            double du = 0.0, dv = 0.0;
            for (int64_t i = 0; i < m; ++i) du = du + u[i] * U[l * m + i];
            for (int64_t c = 0; c < n; ++c) dv = dv + V[l * n + c] * v[c];
            cross = cross + du * dv;
        }
        S2 = S2 + (2.0 * cross + nu2 * nv2);
        r++;
        seen[is] = 1;
        /* reference row residual, moved on once resolved */
        double ui = u[iref], rmax = 0.0;
        for (int64_t c = 0; c < n; ++c) {
            rr[c] = rr[c] - ui * v[c];
            if (fabs(rr[c]) > rmax) rmax = fabs(rr[c]);
        }
        double rlim = rtol * sqrt((S2 > 0.0 ? S2 : 0.0) / (double)m);
        if (!(rmax > rlim)) {
            int64_t in = -1;
            for (int64_t i = 0; i < m; ++i)
                if (!seen[i]) {
                    in = i;
                    break;
                }
            if (in >= 0) {
                iref = in;
                seen[in] = 1;
                rmax = 0.0;
                for (int64_t c = 0; c < n; ++c) {
                    double s = f(ctx, iref, c);
                    for (int l = 0; l < r; ++l) s = s - U[l * m + iref] * V[l * n + c];
                    rr[c] = s;
                    if (fabs(s) > rmax) rmax = fabs(s);
                }
            }
        }
        /* stopping criterion of Alg. 2, with the reference row resolved */
        if (thr >= 0.0 && sqrt(nu2) * sqrt(nv2) <= thr * sqrt(S2 > 0.0 ? S2 : 0.0) &&
            !(rmax > rlim))
            break;
        if (r >= kmax) break;
        /* next column: largest reference-row residual among unused columns */
        int64_t jn = -1;
        double bv = -1.0;
        for (int64_t c = 0; c < n; ++c)
            if (!used[c] && fabs(rr[c]) > bv) {
                bv = fabs(rr[c]);
                jn = c;
            }
        if (jn < 0) break;
        j = jn;
    }
    free(used);
    free(seen);
    free(uh);
    free(rr);
    if (n_rej) *n_rej = rej;
    return r;
}

typedef struct { const double* A; int64_t m; } or_dense_ctx;

static double or_dense_entry(const void* ctx, int64_t i, int64_t j)
{
    const or_dense_ctx* c = (const or_dense_ctx*)ctx;
    return c->A[i + j * c->m];
}

int or_aca_dense(const double* A, int64_t m, int64_t n, double eps, int k_cap,
                 double aca_eta, double eps0, double* U, double* V,
                 int64_t* piv_i, int64_t* piv_j, int64_t* n_rej)
{
    or_dense_ctx c = {A, m};
    return or_aca(or_dense_entry, &c, m, n, eps, k_cap, aca_eta, eps0, U, V,
                  piv_i, piv_j, n_rej);
}

/* ------------------------------------------------------------------------ */
/* The H-matrix: cluster tree, Alg. 1 leaf partition, factors.              */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t tau, sigma; int adm; } or_leaf;

struct or_hmat {
    int64_t N;
    int d, kernel, C, adm_max;
    double ell, sigma2, eta;
    uint64_t* codes;
    int64_t* perm;
    double* coords;      /* Morton order, (N, d) */
    int64_t n_nodes;
    int64_t *lo, *hi;
    double *bbmin, *bbmax;
    or_leaf* adm;
    int64_t n_adm;
    or_leaf* dense;
    int64_t n_dense;
    int32_t* rank;       /* per adm leaf, -1 = not compressed */
    int64_t* rej;
    int64_t* offU;       /* per adm leaf offsets into U, V stores */
    int64_t* offV;
    double *Ust, *Vst;
    int64_t *pivI, *pivJ; /* per adm leaf, rank entries at offP */
    int64_t* offP;
    /* Column side: the set Y2 of A_{phi, Y1 x Y2} (Sec. 6.1 treats two point
     * sets) with its own Morton order and cluster tree. For A_{phi, Y x Y}
     * these point at the row side's arrays (rect = 0). */
    int rect;
    int64_t N2;
    uint64_t* codes2;
    int64_t* perm2;
    double* coords2;     /* Morton order, (N2, d) */
    int64_t n_nodes2;
    int64_t *lo2, *hi2;
    double *bbmin2, *bbmax2;
};

typedef struct { or_leaf* v; int64_t n, cap; } or_leafvec;

static void or_push(or_leafvec* a, int64_t t, int64_t s, int adm)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 1024;
        a->v = (or_leaf*)realloc(a->v, (size_t)a->cap * sizeof(or_leaf));
    }
    a->v[a->n].tau = t;
    a->v[a->n].sigma = s;
    a->v[a->n].adm = adm;
    a->n++;
}

/* Alg. 1 build_block_cluster_tree: split (tau, sigma) into the four child   */
/* pairs iff it is not admissible and both clusters hold more than C_leaf    */
/* indices; otherwise it is a leaf (admissible -> low rank, else dense).     */
/* tau is a node of the row tree, sigma of the column tree (the same tree    */
/* for A_{phi, Y x Y}).                                                      */
static void or_block_tree(const or_hmat* h, int64_t t, int64_t s, double eta2,
                          or_leafvec* adm, or_leafvec* dense)
{
    int d = h->d;
    int a = or_admissible(h->bbmin + t * d, h->bbmax + t * d, h->bbmin2 + s * d,
                          h->bbmax2 + s * d, d, eta2, h->adm_max);
    int64_t nt = h->hi[t] - h->lo[t], ns = h->hi2[s] - h->lo2[s];
    if (!a && nt > h->C && ns > h->C) {
        or_block_tree(h, 2 * t + 1, 2 * s + 1, eta2, adm, dense);
        or_block_tree(h, 2 * t + 1, 2 * s + 2, eta2, adm, dense);
        or_block_tree(h, 2 * t + 2, 2 * s + 1, eta2, adm, dense);
        or_block_tree(h, 2 * t + 2, 2 * s + 2, eta2, adm, dense);
    } else if (a) {
        or_push(adm, t, s, 1);
    } else {
        or_push(dense, t, s, 0);
    }
}

static const or_hmat* or_sort_ctx;

static int or_leaf_cmp(const void* a, const void* b)
{
    const or_leaf* x = (const or_leaf*)a;
    const or_leaf* y = (const or_leaf*)b;
    int64_t xt = or_sort_ctx->lo[x->tau], yt = or_sort_ctx->lo[y->tau];
    if (xt != yt) return xt < yt ? -1 : 1;
    int64_t xs = or_sort_ctx->lo2[x->sigma], ys = or_sort_ctx->lo2[y->sigma];
    if (xs != ys) return xs < ys ? -1 : 1;
    return 0;
}

/* One point set's Morton codes, stable order, Morton-ordered coordinates,   */
/* cluster tree and bounding boxes (Sec. 4.4, 5.1, 2.1, 2.2).               */
static void or_cluster_side(const double* pts, int64_t N, int d, int C, uint64_t** codes,
                            int64_t** perm, double** coords, int64_t* n_nodes, int64_t** lo,
                            int64_t** hi, double** bbmin, double** bbmax)
{
    double blo[3], bhi[3], sc[3];
    *codes = (uint64_t*)malloc((size_t)N * sizeof(uint64_t));
    *perm = (int64_t*)malloc((size_t)N * sizeof(int64_t));
    or_morton(pts, N, d, *codes, blo, bhi, sc);
    or_sort(*codes, N, *perm);
    *coords = (double*)malloc((size_t)N * d * sizeof(double));
    for (int64_t j = 0; j < N; ++j)
        for (int i = 0; i < d; ++i) (*coords)[j * d + i] = pts[(*perm)[j] * d + i];
    *n_nodes = or_tree_nodes(N, C);
    *lo = (int64_t*)malloc((size_t)*n_nodes * sizeof(int64_t));
    *hi = (int64_t*)malloc((size_t)*n_nodes * sizeof(int64_t));
    or_tree_ranges(N, C, *lo, *hi);
    *bbmin = (double*)malloc((size_t)*n_nodes * d * sizeof(double));
    *bbmax = (double*)malloc((size_t)*n_nodes * d * sizeof(double));
    or_bbox(*coords, N, d, C, *lo, *hi, *bbmin, *bbmax);
}

/* Structure of A_{phi, Y1 x Y2}: both sets clustered on their own, then    */
/* Alg. 1 from the pair of roots. pts2 == NULL gives A_{phi, Y x Y}.        */
static or_hmat* or_structure_pair(const double* pts, int64_t N, const double* pts2,
                                  int64_t N2, int d, int kernel, const double* params,
                                  int C, double eta, int adm_max)
{
    or_hmat* h = (or_hmat*)calloc(1, sizeof(or_hmat));
    h->N = N;
    h->d = d;
    h->kernel = kernel;
    h->C = C;
    h->adm_max = adm_max;
    h->ell = params[0];
    h->sigma2 = params[1];
    h->eta = eta;
    or_cluster_side(pts, N, d, C, &h->codes, &h->perm, &h->coords, &h->n_nodes, &h->lo,
                    &h->hi, &h->bbmin, &h->bbmax);
    if (pts2) {
        h->rect = 1;
        h->N2 = N2;
        or_cluster_side(pts2, N2, d, C, &h->codes2, &h->perm2, &h->coords2, &h->n_nodes2,
                        &h->lo2, &h->hi2, &h->bbmin2, &h->bbmax2);
    } else {
        h->N2 = N;
        h->codes2 = h->codes;
        h->perm2 = h->perm;
        h->coords2 = h->coords;
        h->n_nodes2 = h->n_nodes;
        h->lo2 = h->lo;
        h->hi2 = h->hi;
        h->bbmin2 = h->bbmin;
        h->bbmax2 = h->bbmax;
    }

    or_leafvec adm = {0}, dense = {0};
    or_block_tree(h, 0, 0, eta * eta, &adm, &dense);
    or_sort_ctx = h;
    if (adm.n) qsort(adm.v, (size_t)adm.n, sizeof(or_leaf), or_leaf_cmp);
    if (dense.n) qsort(dense.v, (size_t)dense.n, sizeof(or_leaf), or_leaf_cmp);
    h->adm = adm.v;
    h->n_adm = adm.n;
    h->dense = dense.v;
    h->n_dense = dense.n;

    int64_t na = h->n_adm > 0 ? h->n_adm : 1;
    h->rank = (int32_t*)malloc((size_t)na * sizeof(int32_t));
    h->rej = (int64_t*)calloc((size_t)na, sizeof(int64_t));
    for (int64_t b = 0; b < h->n_adm; ++b) h->rank[b] = -1;
    h->offU = (int64_t*)calloc((size_t)na, sizeof(int64_t));
    h->offV = (int64_t*)calloc((size_t)na, sizeof(int64_t));
    h->offP = (int64_t*)calloc((size_t)na, sizeof(int64_t));
    return h;
}

or_hmat* or_build_structure(const double* pts, int64_t N, int d, int kernel,
                            const double* params, int C, double eta, int adm_max)
{
    return or_structure_pair(pts, N, NULL, 0, d, kernel, params, C, eta, adm_max);
}

or_hmat* or_build_structure_rect(const double* pts1, int64_t N1, const double* pts2,
                                 int64_t N2, int d, int kernel, const double* params, int C,
                                 double eta, int adm_max)
{
    return or_structure_pair(pts1, N1, pts2, N2, d, kernel, params, C, eta, adm_max);
}

typedef struct { const or_hmat* h; int64_t t0, s0; } or_block_ctx;

static double or_block_entry(const void* ctx, int64_t i, int64_t j)
{
    const or_block_ctx* c = (const or_block_ctx*)ctx;
    const or_hmat* h = c->h;
    return or_kernel_eval(h->kernel, h->ell, h->coords + (c->t0 + i) * h->d,
                          h->coords2 + (c->s0 + j) * h->d, h->d);
}

/* Threads of the block loops (ACA and the product); 1 = the plain loops.  */
/* The blocks are independent, so ACA gives the same factors on any count; */
/* the product then sums per-thread partial vectors (rounding order only).  */
static int or_threads = 1;
void or_set_threads(int t) { or_threads = t > 1 ? t : 1; }

/* ACA of the admissible leaves ids[0..n) (Alg. 2 per leaf); the factors of  */
/* all listed leaves are kept in one store, appended in list order.          */
void or_compress_ids(or_hmat* h, const int64_t* ids, int64_t n_ids, double aca_eps,
                     int k_cap, double aca_eta, double eps0)
{
    int64_t totU = 0, totV = 0, totP = 0;
    for (int64_t q = 0; q < n_ids; ++q) {
        int64_t b = ids[q];
        int64_t m = h->hi[h->adm[b].tau] - h->lo[h->adm[b].tau];
        int64_t n = h->hi2[h->adm[b].sigma] - h->lo2[h->adm[b].sigma];
        int64_t k = k_cap;
        if (k > m) k = m;
        if (k > n) k = n;
        h->offU[b] = totU;
        h->offV[b] = totV;
        h->offP[b] = totP;
        totU += m * k;
        totV += n * k;
        totP += k;
    }
    free(h->Ust);
    free(h->Vst);
    free(h->pivI);
    free(h->pivJ);
    h->Ust = (double*)malloc((size_t)(totU ? totU : 1) * sizeof(double));
    h->Vst = (double*)malloc((size_t)(totV ? totV : 1) * sizeof(double));
    h->pivI = (int64_t*)malloc((size_t)(totP ? totP : 1) * sizeof(int64_t));
    h->pivJ = (int64_t*)malloc((size_t)(totP ? totP : 1) * sizeof(int64_t));
    for (int64_t b = 0; b < h->n_adm; ++b) h->rank[b] = -1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(or_threads) if (or_threads > 1)
    for (int64_t q = 0; q < n_ids; ++q) {
        int64_t b = ids[q];
        int64_t m = h->hi[h->adm[b].tau] - h->lo[h->adm[b].tau];
        int64_t n = h->hi2[h->adm[b].sigma] - h->lo2[h->adm[b].sigma];
        or_block_ctx c = {h, h->lo[h->adm[b].tau], h->lo2[h->adm[b].sigma]};
        int r = or_aca(or_block_entry, &c, m, n, aca_eps, k_cap, aca_eta, eps0,
                       h->Ust + h->offU[b], h->Vst + h->offV[b], h->pivI + h->offP[b],
                       h->pivJ + h->offP[b], &h->rej[b]);
        h->rank[b] = r;
    }
}

void or_compress_range(or_hmat* h, int64_t b0, int64_t b1, double aca_eps,
                       int k_cap, double aca_eta, double eps0)
{
    int64_t n = b1 > b0 ? b1 - b0 : 0;
    int64_t* ids = (int64_t*)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    for (int64_t q = 0; q < n; ++q) ids[q] = b0 + q;
    or_compress_ids(h, ids, n, aca_eps, k_cap, aca_eta, eps0);
    free(ids);
}

/* Symmetric kernels, phi(y, y') = phi(y', y), give A(sigma, tau) =
 * A(tau, sigma)^T, and the block tree of Alg. 1 holds both leaves. This
 * replaces the factors of every admissible leaf with lo[tau] > lo[sigma] by
 * those of its mirror leaf (sigma, tau) with U and V exchanged, so that the
 * H-matrix is exactly symmetric. Leaves are in (lo[tau], lo[sigma]) order, so
 * the mirror of a leaf is found by binary search. */
void or_mirror_transposed(or_hmat* h)
{
    if (h->rect) return;   /* A_{phi, Y1 x Y2} has no mirror leaves */
    for (int64_t b = 0; b < h->n_adm; ++b) {
        const int64_t tl = h->lo[h->adm[b].tau], sl = h->lo[h->adm[b].sigma];
        if (tl <= sl) continue;
        int64_t a = 0, z = h->n_adm - 1;
        while (a < z) {
            const int64_t mid = (a + z) / 2;
            const int64_t mt = h->lo[h->adm[mid].tau], ms = h->lo[h->adm[mid].sigma];
            if (mt < sl || (mt == sl && ms < tl)) a = mid + 1;
            else z = mid;
        }
        const int64_t mb = a;
        if (h->lo[h->adm[mb].tau] != sl || h->lo[h->adm[mb].sigma] != tl) continue;
        const int64_t m = h->hi[h->adm[b].tau] - tl, n = h->hi[h->adm[b].sigma] - sl;
        const int r = h->rank[mb];
        /* U_b (m x r) = V_mb (its n = m rows), V_b (n x r) = U_mb */
        memcpy(h->Ust + h->offU[b], h->Vst + h->offV[mb], (size_t)m * r * sizeof(double));
        memcpy(h->Vst + h->offV[b], h->Ust + h->offU[mb], (size_t)n * r * sizeof(double));
        for (int l = 0; l < r; ++l) {
            h->pivI[h->offP[b] + l] = h->pivJ[h->offP[mb] + l];
            h->pivJ[h->offP[b] + l] = h->pivI[h->offP[mb] + l];
        }
        h->rank[b] = r;
        h->rej[b] = 0;
    }
}

or_hmat* or_build(const double* pts, int64_t N, int d, int kernel,
                  const double* params, int C, double eta, int adm_max,
                  double aca_eps, int k_cap, double aca_eta, double eps0)
{
    or_hmat* h = or_build_structure(pts, N, d, kernel, params, C, eta, adm_max);
    or_compress_range(h, 0, h->n_adm, aca_eps, k_cap, aca_eta, eps0);
    return h;
}

or_hmat* or_build_rect(const double* pts1, int64_t N1, const double* pts2, int64_t N2,
                       int d, int kernel, const double* params, int C, double eta,
                       int adm_max, double aca_eps, int k_cap, double aca_eta, double eps0)
{
    or_hmat* h = or_build_structure_rect(pts1, N1, pts2, N2, d, kernel, params, C, eta, adm_max);
    or_compress_range(h, 0, h->n_adm, aca_eps, k_cap, aca_eta, eps0);
    return h;
}

void or_free(or_hmat* h)
{
    if (!h) return;
    if (h->rect) {
        free(h->codes2); free(h->perm2); free(h->coords2);
        free(h->lo2); free(h->hi2); free(h->bbmin2); free(h->bbmax2);
    }
    free(h->codes); free(h->perm); free(h->coords);
    free(h->lo); free(h->hi); free(h->bbmin); free(h->bbmax);
    free(h->adm); free(h->dense); free(h->rank); free(h->rej);
    free(h->offU); free(h->offV); free(h->offP);
    free(h->Ust); free(h->Vst); free(h->pivI); free(h->pivJ);
    free(h);
}

int64_t or_n_adm(const or_hmat* h) { return h->n_adm; }
int64_t or_n_dense(const or_hmat* h) { return h->n_dense; }
int64_t or_n_nodes(const or_hmat* h) { return h->n_nodes; }

void or_get_codes(const or_hmat* h, uint64_t* codes)
{
    memcpy(codes, h->codes, (size_t)h->N * sizeof(uint64_t));
}

void or_get_perm(const or_hmat* h, int64_t* perm)
{
    memcpy(perm, h->perm, (size_t)h->N * sizeof(int64_t));
}

void or_get_coords(const or_hmat* h, double* coords_m)
{
    memcpy(coords_m, h->coords, (size_t)h->N * h->d * sizeof(double));
}

void or_get_tree(const or_hmat* h, int64_t* lo, int64_t* hi, double* bbmin, double* bbmax)
{
    memcpy(lo, h->lo, (size_t)h->n_nodes * sizeof(int64_t));
    memcpy(hi, h->hi, (size_t)h->n_nodes * sizeof(int64_t));
    memcpy(bbmin, h->bbmin, (size_t)h->n_nodes * h->d * sizeof(double));
    memcpy(bbmax, h->bbmax, (size_t)h->n_nodes * h->d * sizeof(double));
}

int64_t or_n_cols(const or_hmat* h) { return h->N2; }
int64_t or_n_nodes_cols(const or_hmat* h) { return h->n_nodes2; }

void or_get_col_perm(const or_hmat* h, int64_t* perm)
{
    memcpy(perm, h->perm2, (size_t)h->N2 * sizeof(int64_t));
}

void or_get_col_tree(const or_hmat* h, int64_t* lo, int64_t* hi, double* bbmin, double* bbmax)
{
    memcpy(lo, h->lo2, (size_t)h->n_nodes2 * sizeof(int64_t));
    memcpy(hi, h->hi2, (size_t)h->n_nodes2 * sizeof(int64_t));
    memcpy(bbmin, h->bbmin2, (size_t)h->n_nodes2 * h->d * sizeof(double));
    memcpy(bbmax, h->bbmax2, (size_t)h->n_nodes2 * h->d * sizeof(double));
}

void or_get_adm(const or_hmat* h, int64_t* leaves)
{
    for (int64_t b = 0; b < h->n_adm; ++b) {
        leaves[2 * b] = h->adm[b].tau;
        leaves[2 * b + 1] = h->adm[b].sigma;
    }
}

void or_get_dense(const or_hmat* h, int64_t* leaves)
{
    for (int64_t b = 0; b < h->n_dense; ++b) {
        leaves[2 * b] = h->dense[b].tau;
        leaves[2 * b + 1] = h->dense[b].sigma;
    }
}

void or_get_ranks(const or_hmat* h, int32_t* ranks, int64_t* n_rej)
{
    for (int64_t b = 0; b < h->n_adm; ++b) {
        ranks[b] = h->rank[b];
        if (n_rej) n_rej[b] = h->rej[b];
    }
}

void or_get_factors(const or_hmat* h, int64_t b, double* U, double* V)
{
    int64_t m = h->hi[h->adm[b].tau] - h->lo[h->adm[b].tau];
    int64_t n = h->hi2[h->adm[b].sigma] - h->lo2[h->adm[b].sigma];
    int r = h->rank[b];
    if (r <= 0) return;
    memcpy(U, h->Ust + h->offU[b], (size_t)(m * r) * sizeof(double));
    memcpy(V, h->Vst + h->offV[b], (size_t)(n * r) * sizeof(double));
}

void or_get_pivots(const or_hmat* h, int64_t b, int64_t* piv_i, int64_t* piv_j)
{
    int r = h->rank[b];
    for (int l = 0; l < r; ++l) {
        piv_i[l] = h->pivI[h->offP[b] + l];
        piv_j[l] = h->pivJ[h->offP[b] + l];
    }
}

/* ------------------------------------------------------------------------ */
/* Alg. 3: z|tau += U (V^T x|sigma) on admissible leaves, z|tau += A|tau x   */
/* sigma x|sigma on dense ones. (Alg. 3 prints V^T x|tau; V has |sigma|     */
/* rows, so the product is with x|sigma.) Blocks are visited in canonical   */
/* order; x is permuted into Morton order first (Sec. 5.1) and the result   */
/* permuted back, with sigma^2 x added (Sec. 1, the GPR/KRR variant).        */
/* ------------------------------------------------------------------------ */
static void or_matvec_threads(const or_hmat* h, const double* xm, double* ym);

void or_matvec(const or_hmat* h, const double* x, double* y)
{
    int64_t N = h->N, N2 = h->N2;
    int d = h->d;
    double* xm = (double*)malloc((size_t)(N2 > 0 ? N2 : 1) * sizeof(double));
    double* ym = (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    for (int64_t j = 0; j < N2; ++j) xm[j] = x[h->perm2[j]];
    if (or_threads > 1) {
        or_matvec_threads(h, xm, ym);
        for (int64_t i = 0; i < N; ++i)
            y[h->perm[i]] = h->rect ? ym[i] : ym[i] + h->sigma2 * x[h->perm[i]];
        free(xm);
        free(ym);
        return;
    }
    double* t = (double*)malloc(64 * sizeof(double));
    int tcap = 64;
    for (int64_t b = 0; b < h->n_adm; ++b) {
        int64_t t0 = h->lo[h->adm[b].tau], m = h->hi[h->adm[b].tau] - t0;
        int64_t s0 = h->lo2[h->adm[b].sigma], n = h->hi2[h->adm[b].sigma] - s0;
        int r = h->rank[b];
        if (r <= 0) continue;
        if (r > tcap) {
            tcap = r;
            t = (double*)realloc(t, (size_t)tcap * sizeof(double));
        }
        const double* U = h->Ust + h->offU[b];
        const double* V = h->Vst + h->offV[b];
        for (int l = 0; l < r; ++l) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s = s + V[l * n + j] * xm[s0 + j];
            t[l] = s;
        }
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int l = 0; l < r; ++l) s = s + U[l * m + i] * t[l];
            ym[t0 + i] = ym[t0 + i] + s;
        }
    }
    for (int64_t b = 0; b < h->n_dense; ++b) {
        int64_t t0 = h->lo[h->dense[b].tau], m = h->hi[h->dense[b].tau] - t0;
        int64_t s0 = h->lo2[h->dense[b].sigma], n = h->hi2[h->dense[b].sigma] - s0;
        for (int64_t i = 0; i < m; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j)
                s = s + or_kernel_eval(h->kernel, h->ell, h->coords + (t0 + i) * d,
                                       h->coords2 + (s0 + j) * d, d) * xm[s0 + j];
            ym[t0 + i] = ym[t0 + i] + s;
        }
    }
    /* sigma^2 x on the diagonal only exists for A_{phi, Y x Y} */
    for (int64_t i = 0; i < N; ++i)
        y[h->perm[i]] = h->rect ? ym[i] : ym[i] + h->sigma2 * x[h->perm[i]];
    free(t);
    free(xm);
    free(ym);
}

/* The product's leaf loops on or_threads threads, for timing the oracle on  */
/* all host cores: each thread adds its leaves into a vector of its own and  */
/* the vectors add in thread order (the same leaf terms as or_matvec, summed */
/* in another order).                                                        */
static void or_matvec_threads(const or_hmat* h, const double* xm, double* ym)
{
    int64_t N = h->N;
    int d = h->d;
    int T = or_threads;
    double* part = (double*)calloc((size_t)T * (size_t)(N > 0 ? N : 1), sizeof(double));
#pragma omp parallel num_threads(T)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* yt = part + (size_t)tid * (size_t)(N > 0 ? N : 1);
        int tcap = 64;
        double* t = (double*)malloc((size_t)tcap * sizeof(double));
#pragma omp for schedule(dynamic, 16)
        for (int64_t b = 0; b < h->n_adm; ++b) {
            int64_t t0 = h->lo[h->adm[b].tau], m = h->hi[h->adm[b].tau] - t0;
            int64_t s0 = h->lo2[h->adm[b].sigma], n = h->hi2[h->adm[b].sigma] - s0;
            int r = h->rank[b];
            if (r <= 0) continue;
            if (r > tcap) {
                tcap = r;
                t = (double*)realloc(t, (size_t)tcap * sizeof(double));
            }
            const double* U = h->Ust + h->offU[b];
            const double* V = h->Vst + h->offV[b];
            for (int l = 0; l < r; ++l) {
                double sm = 0.0;
                for (int64_t j = 0; j < n; ++j) sm = sm + V[l * n + j] * xm[s0 + j];
                t[l] = sm;
            }
            for (int64_t i = 0; i < m; ++i) {
                double sm = 0.0;
                for (int l = 0; l < r; ++l) sm = sm + U[l * m + i] * t[l];
                yt[t0 + i] = yt[t0 + i] + sm;
            }
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t b = 0; b < h->n_dense; ++b) {
            int64_t t0 = h->lo[h->dense[b].tau], m = h->hi[h->dense[b].tau] - t0;
            int64_t s0 = h->lo2[h->dense[b].sigma], n = h->hi2[h->dense[b].sigma] - s0;
            for (int64_t i = 0; i < m; ++i) {
                double sm = 0.0;
                for (int64_t j = 0; j < n; ++j)
                    sm = sm + or_kernel_eval(h->kernel, h->ell, h->coords + (t0 + i) * d,
                                             h->coords2 + (s0 + j) * d, d) * xm[s0 + j];
                yt[t0 + i] = yt[t0 + i] + sm;
            }
        }
        free(t);
    }
    for (int tq = 0; tq < T; ++tq)
        for (int64_t i = 0; i < N; ++i) ym[i] = ym[i] + part[(size_t)tq * (size_t)N + i];
    free(part);
}

/* Block-row share of the product (distributed H-matrices, the outlook of   */
/* Sec. 7): the Morton-ordered rows [r0, r1) of y_m = H x_m (+ sigma^2 x_m), */
/* from the Morton-ordered x_m, using only the leaves whose row cluster tau  */
/* meets [r0, r1), in the canonical order of or_matvec. Every leaf that      */
/* touches a row in the range is among them, and each row receives the same  */
/* sums in the same order as in or_matvec, so the rows are bit for bit those */
/* of the whole product.                                                      */
void or_matvec_rows(const or_hmat* h, const double* xm, int64_t r0, int64_t r1, double* yr)
{
    int64_t N = h->N;
    int d = h->d;
    if (r0 < 0) r0 = 0;
    if (r1 > N) r1 = N;
    if (r1 <= r0) return;
    double* ym = (double*)calloc((size_t)(r1 - r0), sizeof(double));
    double* t = (double*)malloc(64 * sizeof(double));
    int tcap = 64;
    for (int64_t b = 0; b < h->n_adm; ++b) {
        int64_t t0 = h->lo[h->adm[b].tau], m = h->hi[h->adm[b].tau] - t0;
        int64_t s0 = h->lo2[h->adm[b].sigma], n = h->hi2[h->adm[b].sigma] - s0;
        int r = h->rank[b];
        if (r <= 0 || t0 + m <= r0 || t0 >= r1) continue;
        if (r > tcap) {
            tcap = r;
            t = (double*)realloc(t, (size_t)tcap * sizeof(double));
        }
        const double* U = h->Ust + h->offU[b];
        const double* V = h->Vst + h->offV[b];
        for (int l = 0; l < r; ++l) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s = s + V[l * n + j] * xm[s0 + j];
            t[l] = s;
        }
        for (int64_t i = 0; i < m; ++i) {
            if (t0 + i < r0 || t0 + i >= r1) continue;
            double s = 0.0;
            for (int l = 0; l < r; ++l) s = s + U[l * m + i] * t[l];
            ym[t0 + i - r0] = ym[t0 + i - r0] + s;
        }
    }
    for (int64_t b = 0; b < h->n_dense; ++b) {
        int64_t t0 = h->lo[h->dense[b].tau], m = h->hi[h->dense[b].tau] - t0;
        int64_t s0 = h->lo2[h->dense[b].sigma], n = h->hi2[h->dense[b].sigma] - s0;
        if (t0 + m <= r0 || t0 >= r1) continue;
        for (int64_t i = 0; i < m; ++i) {
            if (t0 + i < r0 || t0 + i >= r1) continue;
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j)
                s = s + or_kernel_eval(h->kernel, h->ell, h->coords + (t0 + i) * d,
                                       h->coords2 + (s0 + j) * d, d) * xm[s0 + j];
            ym[t0 + i - r0] = ym[t0 + i - r0] + s;
        }
    }
    for (int64_t i = r0; i < r1; ++i)
        yr[i - r0] = h->rect ? ym[i - r0] : ym[i - r0] + h->sigma2 * xm[i];
    free(t);
    free(ym);
}

/* Brute-force truth: y_i = sum_j phi(y_i, y_j) x_j + sigma^2 x_i with       */
/* Neumaier-compensated summation over j.                                    */
static double or_neumaier_row(const double* pts, int64_t N, int d, int kernel,
                              double ell, int64_t i, const double* x)
{
    double s = 0.0, c = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        double term = or_kernel_eval(kernel, ell, pts + i * d, pts + j * d, d) * x[j];
        double t = s + term;
        if (fabs(s) >= fabs(term))
            c = c + ((s - t) + term);
        else
            c = c + ((term - t) + s);
        s = t;
    }
    return s + c;
}

void or_dense_matvec(const double* pts, int64_t N, int d, int kernel,
                     const double* params, const double* x, double* y)
{
    for (int64_t i = 0; i < N; ++i)
        y[i] = or_neumaier_row(pts, N, d, kernel, params[0], i, x) + params[1] * x[i];
}

void or_dense_rows(const double* pts, int64_t N, int d, int kernel,
                   const double* params, const int64_t* rows, int64_t nrows,
                   const double* x, double* y_rows)
{
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        y_rows[r] = or_neumaier_row(pts, N, d, kernel, params[0], i, x) + params[1] * x[i];
    }
}

/* Brute force of A_{phi, Y1 x Y2} x: y_i = sum_j phi(y1_i, y2_j) x_j over  */
/* the N2 points of Y2 (Neumaier-compensated), for the N1 points of Y1.     */
void or_dense_matvec_rect(const double* pts1, int64_t N1, const double* pts2, int64_t N2,
                          int d, int kernel, const double* params, const double* x,
                          double* y)
{
    for (int64_t i = 0; i < N1; ++i) {
        double s = 0.0, c = 0.0;
        for (int64_t j = 0; j < N2; ++j) {
            double v = or_kernel_eval(kernel, params[0], pts1 + i * d, pts2 + j * d, d) * x[j];
            double t = s + v;
            if (fabs(s) >= fabs(v)) c = c + ((s - t) + v);
            else c = c + ((v - t) + s);
            s = t;
        }
        y[i] = s + c;
    }
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradients (Hestenes-Stiefel) on (A_H + sigma^2 I) x = b, the   */
/* system of Sec. 1 solved with the fast H-MVP as the operator.             */
/* ------------------------------------------------------------------------ */
static double or_dot(const double* a, const double* b, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}

int or_cg(const or_hmat* h, const double* b, double* x, double rtol, int maxit,
          double* relres)
{
    if (h->rect) return -1;   /* CG needs the square system A + sigma^2 I */
    int64_t N = h->N;
    double* r = (double*)malloc((size_t)N * sizeof(double));
    double* p = (double*)malloc((size_t)N * sizeof(double));
    double* q = (double*)malloc((size_t)N * sizeof(double));
    or_matvec(h, x, q);
    for (int64_t i = 0; i < N; ++i) {
        r[i] = b[i] - q[i];
        p[i] = r[i];
    }
    double bn = sqrt(or_dot(b, b, N));
    if (bn == 0.0) bn = 1.0;
    double rr = or_dot(r, r, N);
    int it = 0;
    while (it < maxit && sqrt(rr) / bn > rtol) {
        or_matvec(h, p, q);
        double alpha = rr / or_dot(p, q, N);
        for (int64_t i = 0; i < N; ++i) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
        }
        double rr1 = or_dot(r, r, N);
        double beta = rr1 / rr;
        for (int64_t i = 0; i < N; ++i) p[i] = r[i] + beta * p[i];
        rr = rr1;
        it++;
    }
    *relres = sqrt(rr) / bn;
    free(r);
    free(p);
    free(q);
    return it;
}

/* ------------------------------------------------------------------------ */
/* Learned rank model (not in the paper): features of an admissible block   */
/* (tau, sigma) with l the kernel length scale:                              */
/*   f0 = d/3, f1 = log2|tau|/16, f2 = log2|sigma|/16,                       */
/*   f3 = log2(1 + diam(Q_tau)/l), f4 = log2(1 + diam(Q_sigma)/l),           */
/*   f5 = log2(1 + dist(Q_tau,Q_sigma)/l), f6 = -log10(eps)/8, f7 = kernel.  */
/* ------------------------------------------------------------------------ */
void or_block_features(const or_hmat* h, double aca_eps, double* feats)
{
    int d = h->d;
    for (int64_t b = 0; b < h->n_adm; ++b) {
        int64_t t = h->adm[b].tau, s = h->adm[b].sigma;
        double Dt = 0.0, Ds = 0.0, G2 = 0.0;
        for (int i = 0; i < d; ++i) {
            double et = h->bbmax[t * d + i] - h->bbmin[t * d + i];
            double es = h->bbmax2[s * d + i] - h->bbmin2[s * d + i];
            Dt = Dt + et * et;
            Ds = Ds + es * es;
            double g1 = h->bbmin[t * d + i] - h->bbmax2[s * d + i];
            double g2 = h->bbmin2[s * d + i] - h->bbmax[t * d + i];
            if (g1 < 0.0) g1 = 0.0;
            if (g2 < 0.0) g2 = 0.0;
            G2 = G2 + (g1 * g1 + g2 * g2);
        }
        double* f = feats + b * 8;
        f[0] = d / 3.0;
        f[1] = log2((double)(h->hi[t] - h->lo[t])) / 16.0;
        f[2] = log2((double)(h->hi2[s] - h->lo2[s])) / 16.0;
        f[3] = log2(1.0 + sqrt(Dt) / h->ell);
        f[4] = log2(1.0 + sqrt(Ds) / h->ell);
        f[5] = log2(1.0 + sqrt(G2) / h->ell);
        f[6] = -log10(aca_eps) / 8.0;
        f[7] = (double)h->kernel;
    }
}

/* MLP 8 -> 64 -> 64 -> 1 with ReLU: h1 = relu(W1 f + b1), h2 = relu(W2 h1 + */
/* b2), yhat = W3 h2 + b3. Loss = mean over samples of (yhat - target)^2.   */
#define OR_H 64
#define OR_F 8
static void or_mlp_unpack(const double* th, const double** W1, const double** b1,
                          const double** W2, const double** b2, const double** W3,
                          const double** b3)
{
    *W1 = th;
    *b1 = *W1 + OR_H * OR_F;
    *W2 = *b1 + OR_H;
    *b2 = *W2 + OR_H * OR_H;
    *W3 = *b2 + OR_H;
    *b3 = *W3 + OR_H;
}

static double or_mlp_one(const double* th, const double* f, double* h1, double* h2)
{
    const double *W1, *b1, *W2, *b2, *W3, *b3;
    or_mlp_unpack(th, &W1, &b1, &W2, &b2, &W3, &b3);
    for (int o = 0; o < OR_H; ++o) {
        double s = b1[o];
        for (int i = 0; i < OR_F; ++i) s = s + W1[o * OR_F + i] * f[i];
        h1[o] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < OR_H; ++o) {
        double s = b2[o];
        for (int i = 0; i < OR_H; ++i) s = s + W2[o * OR_H + i] * h1[i];
        h2[o] = s > 0.0 ? s : 0.0;
    }
    double y = b3[0];
    for (int i = 0; i < OR_H; ++i) y = y + W3[i] * h2[i];
    return y;
}

void or_mlp_forward(const double* theta, const double* F, int64_t n, double* out)
{
    double h1[OR_H], h2[OR_H];
    for (int64_t s = 0; s < n; ++s) out[s] = or_mlp_one(theta, F + s * OR_F, h1, h2);
}

double or_mlp_loss_grad(const double* theta, const double* F, const double* target,
                        int64_t n, double* grad)
{
    const double *W1, *b1, *W2, *b2, *W3, *b3;
    or_mlp_unpack(theta, &W1, &b1, &W2, &b2, &W3, &b3);
    if (grad) memset(grad, 0, OR_MLP_NPARAM * sizeof(double));
    double *gW1 = grad, *gb1 = grad + OR_H * OR_F, *gW2 = gb1 + OR_H;
    double *gb2 = gW2 + OR_H * OR_H, *gW3 = gb2 + OR_H, *gb3 = gW3 + OR_H;
    double loss = 0.0;
    double h1[OR_H], h2[OR_H], d1[OR_H], d2[OR_H];
    for (int64_t s = 0; s < n; ++s) {
        const double* f = F + s * OR_F;
        double y = or_mlp_one(theta, f, h1, h2);
        double e = y - target[s];
        loss = loss + e * e;
        if (!grad) continue;
        double dy = 2.0 * e / (double)n;
        gb3[0] = gb3[0] + dy;
        for (int i = 0; i < OR_H; ++i) {
            gW3[i] = gW3[i] + dy * h2[i];
            d2[i] = h2[i] > 0.0 ? dy * W3[i] : 0.0;
        }
        for (int o = 0; o < OR_H; ++o) {
            gb2[o] = gb2[o] + d2[o];
            for (int i = 0; i < OR_H; ++i) gW2[o * OR_H + i] = gW2[o * OR_H + i] + d2[o] * h1[i];
        }
        for (int i = 0; i < OR_H; ++i) {
            double s2 = 0.0;
            for (int o = 0; o < OR_H; ++o) s2 = s2 + W2[o * OR_H + i] * d2[o];
            d1[i] = h1[i] > 0.0 ? s2 : 0.0;
        }
        for (int o = 0; o < OR_H; ++o) {
            gb1[o] = gb1[o] + d1[o];
            for (int i = 0; i < OR_F; ++i) gW1[o * OR_F + i] = gW1[o * OR_F + i] + d1[o] * f[i];
        }
    }
    return loss / (double)n;
}

/* Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;     */
/* theta -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).                */
void or_adam_step(double* theta, const double* grad, double* m, double* v,
                  int64_t n, int64_t t, double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)t);
    double c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        theta[i] = theta[i] - lr * mh / (sqrt(vh) + eps);
    }
}
