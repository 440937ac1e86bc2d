// hm_api.cu -- the C-ABI of libhm.so (include/hm.h): handle life cycle, the
// build pipeline, the product, statistics, exports and conjugate gradients.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <unordered_map>
#include <mutex>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "hm_build.cuh"
#include "hm_handle.cuh"

namespace hm {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void check_cuda(cudaError_t e, const char* what, const char* file, int line)
{
    if (e == cudaSuccess) return;
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                      std::to_string(line) + ")";
    throw Error(e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA, msg);
}

void fail(int code, const std::string& msg) { throw Error(code, msg); }

void set_error(const std::string& s) { g_last_error = s; }

int to_status(const std::exception& e)
{
    if (auto* he = dynamic_cast<const Error*>(&e)) {
        set_error(he->what());
        return he->code;
    }
    if (dynamic_cast<const std::bad_alloc*>(&e)) {
        set_error("host allocation failed");
        return HM_ENOMEM;
    }
    set_error(e.what());
    return HM_ECUDA;
}

// ------------------------------------------------------------------ memory
static bool g_pool_ready = false;
// test hook: the n-th device allocation from now fails (0: none)
static std::atomic<int64_t> g_fail_alloc{0};
// device bytes the library holds (hm_device_bytes)
static std::mutex g_live_mu;
static std::unordered_map<void*, size_t> g_live;
static uint64_t g_live_bytes = 0;

void* dev_alloc(size_t bytes, cudaStream_t s)
{
    if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1)
        fail(HM_ENOMEM, "device allocation of " + std::to_string(bytes) +
                            " bytes failed (injected by the test hook)");
    if (!g_pool_ready) {
        int dev = 0;
        HM_CUDA(cudaGetDevice(&dev));
        cudaMemPool_t pool;
        HM_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
        uint64_t thr = UINT64_MAX;  // keep freed blocks cached in this process
        HM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pool_ready = true;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(HM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                            cudaGetErrorString(e));
    }
    if (p) {
        std::lock_guard<std::mutex> lk(g_live_mu);
        g_live[p] = bytes;
        g_live_bytes += bytes;
    }
    return p;
}

void dev_free(void* p, cudaStream_t s)
{
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        auto it = g_live.find(p);
        if (it != g_live.end()) {
            g_live_bytes -= it->second;
            g_live.erase(it);
        }
    }
    cudaFreeAsync(p, s);
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    if (bytes) HM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

void copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    if (bytes) HM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

static std::atomic<uint64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int num_sms()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        HM_CUDA(cudaGetDevice(&dev));
        HM_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    }
    return n;
}

KernelParams make_kernel_params(int kernel, double ell)
{
    KernelParams k;
    k.kernel = kernel;
    k.c64 = kernel == HM_GAUSSIAN ? 1.0 / (ell * ell)
          : kernel == HM_MATERN32 ? std::sqrt(3.0) / ell
                                  : 0.25 / (ell * ell);
    k.c32 = (float)k.c64;
    return k;
}

}  // namespace hm

using namespace hm;

// ------------------------------------------------------------------ C ABI
extern "C" {

void hm_options_default(hm_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = HM_PREC_FP64;
    o->near_format = HM_NEAR_AUTO;
    o->adm_max = 0;
    o->k_cap = 64;
    o->aca_eta = 0.0;
    o->eps0 = 0.0;
    o->accumulate = 0;
    o->rank_model = 0;
    o->rank_model_theta = nullptr;
    o->scratch_gb = 0.0;
    o->stream = nullptr;
}

const char* hm_last_error(void) { return g_last_error.c_str(); }

uint64_t hm_kernel_launches(void) { return g_launches.load(); }

int hm_set_gather_shape(int shape)
{
    set_error("");
    const int r = hm::mvp_force_shape(shape);
    if (r != HM_OK) set_error("gather shape must be -1 (tuned) or 0 .. 4");
    return r;
}

int hm_set_aca_shape(int cls, int shape)
{
    set_error("");
    if (cls < -1 || cls >= hm::ACA_NCLASS || shape < -1 || shape > 2) {
        set_error("ACA shape: class -1 or 0 .. 11, shape -1 .. 2");
        return HM_EINVAL;
    }
    for (int c = (cls < 0 ? 0 : cls); c < (cls < 0 ? hm::ACA_NCLASS : cls + 1); ++c)
        hm::set_aca_shape(c, shape);
    return HM_OK;
}

int hm_tune_aca_shapes(const double* points, int64_t N, int d, int kernel, const double* params,
                       int leaf_size, double eta, double aca_eps, const hm_options* opt,
                       int reps, int* shapes)
{
    set_error("");
    int saved[hm::ACA_NCLASS];
    for (int c = 0; c < hm::ACA_NCLASS; ++c) saved[c] = hm::aca_shape(c);
    try {
        hm_options o;
        hm_options_default(&o);
        if (opt) o = *opt;
        if (o.on_the_fly) fail(HM_EINVAL, "ACA shape tuning builds stored factors (on_the_fly = 0)");
        if (reps < 1) reps = 1;
        o.profile = 2;   // size classes one after another: one time per class
        constexpr int NS = 3;
        double t[NS][hm::ACA_NCLASS];
        for (int sh = 0; sh < NS; ++sh) {
            for (int c = 0; c < hm::ACA_NCLASS; ++c) {
                t[sh][c] = -1.0;
                hm::set_aca_shape(c, sh);
            }
            for (int r = 0; r < reps; ++r) {
                std::unique_ptr<hm_handle_s> h(new hm_handle_s());
                int64_t Ns[1] = {N};
                int ds[1] = {d};
                build_sets(*h, 1, points, Ns, ds, kernel, params, leaf_size, eta, aca_eps, o);
                for (int c = 0; c < hm::ACA_NCLASS; ++c) {
                    const double v = h->stats.t_aca_class_ms[c];
                    if (v > 0.0 && (t[sh][c] < 0.0 || v < t[sh][c])) t[sh][c] = v;
                }
            }
        }
        for (int c = 0; c < hm::ACA_NCLASS; ++c) {
            int best = -1;
            for (int sh = 0; sh < NS; ++sh)
                if (t[sh][c] > 0.0 && (best < 0 || t[sh][c] < t[best][c])) best = sh;
            hm::set_aca_shape(c, best);    // -1 (the default) for an empty class
            if (shapes) shapes[c] = best;
        }
        return HM_OK;
    } catch (const std::exception& e) {
        for (int c = 0; c < hm::ACA_NCLASS; ++c) hm::set_aca_shape(c, saved[c]);
        return to_status(e);
    }
}

int hm_set_batch_limits(int64_t aca_entries, int64_t gather_items)
{
    set_error("");
    if (aca_entries < 0 || gather_items < 0) {
        set_error("batch limits must be >= 0");
        return HM_EINVAL;
    }
    hm::set_batch_limits(aca_entries, gather_items);
    return HM_OK;
}

int hm_set_test_hook(int hook, int64_t value)
{
    set_error("");
    switch (hook) {
    case HM_HOOK_ACA_STEP_LIMIT:
        if (value < 0 || value > INT32_MAX) break;
        hm::set_aca_step_limit((int)value);
        return HM_OK;
    case HM_HOOK_WAIT_LIMIT_NS:
        if (value < 0) break;
        hm::set_mvp_wait_ns((uint64_t)value);
        return HM_OK;
    case HM_HOOK_GATHER_WITHHOLD:
        if (value < 0 || value > INT32_MAX) break;
        hm::set_mvp_withhold((int)value - 1);
        return HM_OK;
    case HM_HOOK_FAIL_ALLOC:
        if (value < 0) break;
        g_fail_alloc = value;
        return HM_OK;
    case HM_HOOK_TRAVERSAL_KAPPA:
        if (value < 0 || value > (1 << 20)) break;
        hm::set_traversal_kappa(value);
        return HM_OK;
    case HM_HOOK_TRAVERSAL_TRIES:
        if (value < 0 || value > 64) break;
        hm::set_traversal_attempts((int)value);
        return HM_OK;
    default:
        break;
    }
    set_error("unknown test hook or value out of range");
    return HM_EINVAL;
}

hm_handle hm_build_ex(const double* points, int64_t N, int d, int kernel, const double* params,
                      int leaf_size, double eta, double aca_eps, const hm_options* opt,
                      int* status)
{
    set_error("");
    try {
        hm_options o;
        hm_options_default(&o);
        if (opt) o = *opt;
        std::unique_ptr<hm_handle_s> h(new hm_handle_s());
        int64_t Ns[1] = {N};
        int ds[1] = {d};
        build_sets(*h, 1, points, Ns, ds, kernel, params, leaf_size, eta, aca_eps, o);
        if (status) *status = HM_OK;
        return h.release();
    } catch (const std::exception& e) {
        int st = to_status(e);
        if (status) *status = st;
        return nullptr;
    }
}

hm_handle hm_build_rect(const double* rows, int64_t N1, const double* cols, int64_t N2, int d,
                        int kernel, const double* params, int leaf_size, double eta,
                        double aca_eps, const hm_options* opt, int* status)
{
    set_error("");
    try {
        hm_options o;
        hm_options_default(&o);
        if (opt) o = *opt;
        if (!rows || !cols) fail(HM_EINVAL, "points is NULL");
        if (N1 < 1 || N2 < 1) fail(HM_EINVAL, "N must be >= 1");
        if (d < 1 || d > 3) fail(HM_EINVAL, "d must be 1, 2 or 3");
        if (N1 + N2 >= (1ll << 31)) fail(HM_EINVAL, "more than 2^31 points");
        std::unique_ptr<hm_handle_s> h(new hm_handle_s());
        // both sets in one device array, rows first (the build reads them there)
        cudaStream_t s = (cudaStream_t)o.stream;
        DevBuf<double> both((N1 + N2) * d, s);
        copy_in(both.p, rows, N1 * d * sizeof(double), s);
        copy_in(both.p + N1 * d, cols, N2 * d * sizeof(double), s);
        int64_t Ns[2] = {N1, N2};
        int ds[2] = {d, d};
        build_sets(*h, 2, both.p, Ns, ds, kernel, params, leaf_size, eta, aca_eps, o, true);
        HM_CUDA(cudaStreamSynchronize(s));
        if (status) *status = HM_OK;
        return h.release();
    } catch (const std::exception& e) {
        int st = to_status(e);
        if (status) *status = st;
        return nullptr;
    }
}

hm_handle hm_build(const double* points, int64_t N, int d, int kernel, const double* params,
                   int leaf_size, double eta, double aca_eps)
{
    return hm_build_ex(points, N, d, kernel, params, leaf_size, eta, aca_eps, nullptr, nullptr);
}

int hm_matvec_ex(hm_handle h, const double* x, double* y, int nrhs, void* stream)
{
    set_error("");
    try {
        if (!h) fail(HM_EINVAL, "null handle");
        if (!x || !y || nrhs < 1) fail(HM_EINVAL, "bad matvec arguments");
        matvec(*h, x, y, nrhs, stream ? (cudaStream_t)stream : h->stream);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_matvec(hm_handle h, const double* x, double* y)
{
    return hm_matvec_ex(h, x, y, 1, nullptr);
}

uint64_t hm_device_bytes(void)
{
    std::lock_guard<std::mutex> lk(g_live_mu);
    return g_live_bytes;
}

int hm_check_status(hm_handle h)
{
    set_error("");
    try {
        if (!h) fail(HM_EINVAL, "null handle");
        int st = 0;
        HM_CUDA(cudaMemcpyAsync(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        HM_CUDA(cudaStreamSynchronize(h->stream));
        if (st) {
            HM_CUDA(cudaMemsetAsync(h->status.p, 0, sizeof(int), h->stream));
            HM_CUDA(cudaStreamSynchronize(h->stream));
            fail(HM_ETIMEOUT, std::string("a device loop or wait gave up (status ") +
                                  std::to_string(st) + ")");
        }
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

void hm_free(hm_handle h)
{
    if (!h) return;
    try {
        cudaStream_t s = h->stream;
        delete h;
        cudaStreamSynchronize(s);
    } catch (...) {
    }
}

int hm_get_stats(hm_handle h, hm_stats* out)
{
    set_error("");
    if (!h || !out) {
        set_error("null argument");
        return HM_EINVAL;
    }
    try {
        if (h->opt.profile && h->opt.on_the_fly) {
            // the on-the-fly product keeps its sums in the stats themselves
            *out = h->stats;
            h->stats.mvp_count = 0;
            h->stats.t_mvp_ms = h->stats.t_np_aca_ms = h->stats.t_np_lowrank_ms = 0.0;
            h->stats.t_np_near_ms = 0.0;
            return HM_OK;
        }
        if (h->opt.profile) {
            h->timer.collect();
            h->stats.mvp_count = h->timer.count;
            h->stats.t_mvp_ms = h->timer.t_total;
            h->stats.t_mvp_gather_ms = h->timer.t_gather;
            h->stats.t_mvp_vtx_ms = h->timer.t_vtx;
            h->stats.t_mvp_tile_ms = h->timer.t_tile;
            h->stats.t_mvp_tail_ms = h->timer.t_tail;
            h->timer.count = 0;
            h->timer.t_total = h->timer.t_gather = h->timer.t_vtx = h->timer.t_tile = 0.0;
            h->timer.t_tail = 0.0;
        }
    } catch (const std::exception& e) {
        return to_status(e);
    }
    *out = h->stats;
    return HM_OK;
}

int hm_export_structure(hm_handle h, uint64_t* codes, int64_t* perm, int64_t* adm,
                        int64_t* dense, int32_t* ranks)
{
    set_error("");
    try {
        if (!h) fail(HM_EINVAL, "null handle");
        export_structure(*h, codes, perm, adm, dense, ranks);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_export_tree(hm_handle h, int64_t* lo, int64_t* hi, double* bbmin, double* bbmax)
{
    set_error("");
    try {
        if (!h) fail(HM_EINVAL, "null handle");
        export_tree(*h, lo, hi, bbmin, bbmax);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_export_factors(hm_handle h, int64_t b, double* U, double* V, int* rank)
{
    set_error("");
    try {
        if (!h) fail(HM_EINVAL, "null handle");
        export_factors(*h, b, U, V, rank);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_cg(hm_handle h, const double* b, double* x, double rtol, int maxit, int* iters,
          double* relres)
{
    set_error("");
    try {
        if (!h || !b || !x) fail(HM_EINVAL, "null argument");
        if (maxit < 0) fail(HM_EINVAL, "maxit < 0");
        cg_solve(*h, b, x, rtol, maxit, iters, relres);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_morton_codes(const double* points, int64_t N, int d, uint64_t* codes, void* stream)
{
    set_error("");
    try {
        if (!points || !codes || N < 1 || d < 1 || d > 3) fail(HM_EINVAL, "bad arguments");
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf<double> box(9, s);
        morton_codes(points, N, d, codes, nullptr, box.p, s);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_radix_sort_pairs(uint64_t* keys, uint32_t* values, int64_t n, int key_bits, void* stream)
{
    set_error("");
    try {
        if (!keys || !values || n < 0 || key_bits < 0 || key_bits > 64)
            fail(HM_EINVAL, "bad arguments");
        radix_sort_u64_u32(keys, values, n, key_bits, (cudaStream_t)stream);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_radix_sort_pairs_noalloc(uint64_t* keys, uint32_t* values, int64_t n, int key_bits,
                                void* stream)
{
    set_error("");
    try {
        if (!keys || !values || n < 0 || key_bits < 0 || key_bits > 64)
            fail(HM_EINVAL, "bad arguments");
        if (n > HM_NOALLOC_SORT_MAX)
            fail(HM_EINVAL, "n = " + std::to_string(n) + " exceeds HM_NOALLOC_SORT_MAX (" +
                                std::to_string((long long)HM_NOALLOC_SORT_MAX) + ")");
        if (n > 1 && (!is_device_ptr(keys) || !is_device_ptr(values)))
            fail(HM_EINVAL, "keys and values must be device pointers");
        radix_sort_noalloc(keys, values, n, key_bits, (cudaStream_t)stream);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

int hm_alu_peak(int precision, double* flops)
{
    set_error("");
    try {
        if (!flops) fail(HM_EINVAL, "flops is NULL");
        if (precision != HM_PREC_FP64 && precision != HM_PREC_MIXED)
            fail(HM_EINVAL, "unknown precision");
        *flops = alu_peak(precision);
        return HM_OK;
    } catch (const std::exception& e) {
        return to_status(e);
    }
}

}  // extern "C"
