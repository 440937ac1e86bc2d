// hm_handle.cuh -- the handle behind hm_handle / hm_batch and the pipeline
// functions that the C-ABI entry points call.
#pragma once

#include <memory>
#include <vector>

#include "hm_build.cuh"

namespace hm {

struct FactorSegment {
    DevBuf<char> mem;
};

}  // namespace hm

struct hm_handle_s {
    int sym_near = 0;                 // symmetric near field (hm_options.symmetric = 2)
    hm_options opt{};
    int kernel = 0, leaf = 0, precision = 0, near_format = 0;
    double ell = 1.0, sigma2 = 0.0, eta = 0.0, aca_eps = 0.0;
    cudaStream_t stream = 0;
    hm::KernelParams kp{};
    std::vector<hm::SetStructure> sets;
    int64_t Ntot = 0, n_nodes_tot = 0, n_adm = 0, n_dense = 0, n_tiles = 0;
    int64_t max_set_n = 0;
    int64_t factor_entries_U = 0;   // sum_b k_b m_b
    int64_t factor_entries_Vc = 0;  // sum over canonical blocks (row0 < col0) of k_b n_b
    // A_{phi, Y1 x Y2}: set 0 gives the rows, set 1 the columns; the product
    // runs on staging vectors of Ntot entries (x in set 1's part, zeros in
    // set 0's; y in set 0's part)
    bool rect = false;
    int64_t n_rows = 0, n_cols = 0;
    double rect_fro2 = 0.0;   // mixed precision: sum of ||A_b||_F^2 over the dense leaves
    hm::DevBuf<double> rxbuf, rybuf;
    // points and structure
    hm::DevBuf<double> X64;
    hm::DevBuf<float> X32;
    hm::DeviceCoords X;
    hm::DevBuf<int64_t> perm;
    hm::DevBuf<uint64_t> codes;
    hm::DevBuf<int32_t> node_lo, node_hi;
    hm::DevBuf<double> bmin, bmax;
    hm::DevBuf<int2> adm_pairs, dense_pairs;   // set-local node ids, canonical order
    hm::DevBuf<int32_t> adm_set, dense_set;     // owning set of each leaf
    hm::DevBuf<hm::Blk> ablk, dblk;
    hm::DevBuf<int64_t> tile_row0;
    hm::DevBuf<int32_t> tile_m;
    // factors
    hm::DevBuf<int32_t> kres, rank, nrej, flags;
    hm::DevBuf<uint64_t> Uptr, Vptr;   // per block (U: valid until the relayout)
    std::vector<std::unique_ptr<hm::FactorSegment>> usegments, vsegments;
    hm::DevBuf<char> ustore;            // tile-major U slices
    // near field (tile-major slices)
    hm::DevBuf<char> near;
    // host copies of the gather lists for factor export (filled on demand)
    std::vector<int2> h_lr_ent;
    std::vector<hm::LrDesc> h_lr_desc;
    std::vector<int32_t> h_lr_tile, h_tile_m;
    // product
    hm::MvpLists lists;
    hm::MvpPlan plan;
    hm::MvpWork work;
    hm::MvpTimer timer;
    hm::DevBuf<double> xbuf, ybuf;
    // on-the-fly product: passes of consecutive admissible leaves
    // [np_pass[q], np_pass[q + 1]), their ids, the factor scratch, t of a
    // pass (np_kcap entries per leaf), the permuted x and the row sums
    std::vector<int64_t> np_pass;
    hm::DevBuf<uint32_t> np_ids;
    hm::DevBuf<char> np_scratch, np_t, np_xm;
    hm::DevBuf<double> np_yacc, np_part;   // row sums; near-field item sums
    int np_kcap = 0, np_ld = 0;             // t entries per leaf; rows per item sum
    hm::DevBuf<int32_t> np_kpred;           // rank model: predicted ranks per leaf
    int64_t np_mispredicted = 0;            // re-run blocks, summed over products
    // V^T x items and apply items of the low-rank part, the t partials of a
    // pass and the apply items' running row sums
    hm::DevBuf<int64_t> np_vptr, np_aptr;
    hm::DevBuf<int2> np_vitems;
    hm::DevBuf<int3> np_aitems;
    std::vector<int64_t> np_hvptr;
    int64_t np_naitems = 0;
    hm::DevBuf<char> np_tp;
    hm::DevBuf<double> np_acc;
    // symmetric on-the-fly handles: pass q compresses the canonical leaves of
    // its block range (np_ids[np_cptr[q] ..)) and applies them and their
    // mirror leaves; np_passid / np_tidx give every leaf its pass and its
    // place in the pass's block list np_pblk[np_pbptr[q] ..), whose V^T x
    // items are np_pitems[np_piptr[q] ..) (leaf b's first at np_pfirst[b])
    std::vector<int64_t> np_cptr, np_pbptr, np_piptr;
    hm::DevBuf<int32_t> np_passid, np_tidx;
    hm::DevBuf<int64_t> np_pblk, np_pfirst, np_pitems;
    hm::DevBuf<int> status;
    hm_stats stats{};
    ~hm_handle_s();
};

struct hm_batch_s {
    hm_handle_s h;
    std::vector<int64_t> set_n;
    std::vector<int> set_d;
};

namespace hm {

void set_error(const std::string& s);
int to_status(const std::exception& e);

void build_sets(hm_handle_s& h, int nsets, const double* points_all, const int64_t* N,
                const int* d, int kernel, const double* params, int leaf, double eta,
                double aca_eps, const hm_options& opt, bool rect = false);
void matvec(hm_handle_s& h, const double* x, double* y, int nrhs, cudaStream_t s);
// The product of an on-the-fly handle (device x, y; one vector).
void np_matvec(hm_handle_s& h, const double* x, double* y, int accumulate, cudaStream_t s);
void export_structure(hm_handle_s& h, uint64_t* codes, int64_t* perm, int64_t* adm,
                      int64_t* dense, int32_t* ranks);
void export_tree(hm_handle_s& h, int64_t* lo, int64_t* hi, double* bbmin, double* bbmax);
void export_factors(hm_handle_s& h, int64_t b, double* U, double* V, int* rank);
void add_perm_offsets(hm_handle_s& h);
void fill_block_sets(hm_handle_s& h);
void alloc_factor_meta(hm_handle_s& h);
void compress(hm_handle_s& h, const uint32_t* ids, int64_t n, const int32_t* kpred,
              bool keep_reserved = false);
// learned rank model (hm_mlp.cu)
// Predicted ranks (the rank model) of the admissible blocks ids[0..nids)
// into kpred[id] (all blocks when ids is null).
void predict_ranks(hm_handle_s& h, int32_t* kpred, const uint32_t* ids = nullptr,
                   int64_t nids = -1);
void rerun_mispredicted(hm_handle_s& h);
void cg_solve(hm_handle_s& h, const double* b, double* x, double rtol, int maxit, int* iters,
              double* relres);

}  // namespace hm
