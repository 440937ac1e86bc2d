// hm_aca.cu -- batched ACA (Alg. 2, Sec. 5.4.1): dispatch of every size class
// and rank bucket to the team kernels (hm_aca_team.cuh, instantiated in
// hm_aca_team_f.cu / hm_aca_team_d.cu / hm_aca_k1.cu) or to the cluster
// kernels of hm_aca_impl.cuh, which this unit instantiates for the Gaussian
// and Matern-3/2 kernels.
#include <atomic>

#include "hm_aca_impl.cuh"

namespace hm {

namespace {
std::atomic<int> g_aca_shape[ACA_NCLASS];
std::atomic<int> g_aca_step_limit{0};
struct ShapeInit {
    ShapeInit()
    {
        for (int c = 0; c < ACA_NCLASS; ++c) g_aca_shape[c] = -1;
    }
} g_shape_init;
}  // namespace

int aca_shape(int cls) { return g_aca_shape[cls].load(); }
int aca_default_shape(int cls) { return cls <= 8 ? 1 : 0; }
int aca_step_limit() { return g_aca_step_limit.load(); }

namespace {
std::atomic<int64_t> g_aca_batch{0}, g_mvp_batch{0};
}  // namespace

int64_t aca_batch_entries() { return g_aca_batch.load(); }
int64_t mvp_batch_items() { return g_mvp_batch.load(); }
void set_batch_limits(int64_t aca_entries, int64_t gather_items)
{
    g_aca_batch = aca_entries;
    g_mvp_batch = gather_items;
}
void set_aca_shape(int cls, int shape) { g_aca_shape[cls] = shape; }
void set_aca_step_limit(int v) { g_aca_step_limit = v; }

void aca_run(int precision, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
             const uint32_t* order, int64_t n, int cls, int kb, int64_t max_n, cudaStream_t s)
{
    if (n <= 0) return;
    if (a.k_cap > KBUF) fail(HM_ENOTSUP, "k_cap above 128 is not supported");
    const bool f64 = precision == HM_PREC_FP64;
    int shape = aca_shape(cls);
    if (shape < 0) shape = aca_default_shape(cls);
    if (kb < ACA_NKB - 1 && shape > 0) {
        const int KT = 16 << kb;
        auto team = [&](int sh) {
            return kp.kernel == HM_MATERN_K1
                       ? aca_team_k1(f64, kp, X, a, order, n, cls, sh, KT, s)
                       : aca_team_gm(f64, kp, X, a, order, n, cls, sh, KT, s);
        };
        // an alternative shape not compiled for this kernel runs the default
        if (team(shape) || (shape > 1 && team(1))) return;
    }
    if (kp.kernel == HM_GAUSSIAN) {
        if (f64) launch_all<double, HM_GAUSSIAN>(kp, X, a, order, n, cls, max_n, s);
        else launch_all<float, HM_GAUSSIAN>(kp, X, a, order, n, cls, max_n, s);
    } else if (kp.kernel == HM_MATERN32) {
        if (f64) launch_all<double, HM_MATERN32>(kp, X, a, order, n, cls, max_n, s);
        else launch_all<float, HM_MATERN32>(kp, X, a, order, n, cls, max_n, s);
    } else {
        aca_run_k1(f64, kp, X, a, order, n, cls, kb, max_n, s);
    }
}

}  // namespace hm
