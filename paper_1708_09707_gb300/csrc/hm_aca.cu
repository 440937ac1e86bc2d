// hm_aca.cu -- batched ACA (Alg. 2, Sec. 5.4.1) for the Gaussian and
// Matern-3/2 kernels; the Matern kernel of order 1 is instantiated in
// hm_aca_k1.cu. The kernels themselves are in hm_aca_impl.cuh.
#include "hm_aca_impl.cuh"

namespace hm {

void aca_run(int precision, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
             const uint32_t* order, int64_t n, int cls, int64_t max_n, cudaStream_t s)
{
    if (n <= 0) return;
    if (a.k_cap > KBUF) fail(HM_ENOTSUP, "k_cap above 128 is not supported");
    const bool f64 = precision == HM_PREC_FP64;
    if (kp.kernel == HM_GAUSSIAN) {
        if (f64) launch_all<double, HM_GAUSSIAN>(kp, X, a, order, n, cls, max_n, s);
        else launch_all<float, HM_GAUSSIAN>(kp, X, a, order, n, cls, max_n, s);
    } else if (kp.kernel == HM_MATERN32) {
        if (f64) launch_all<double, HM_MATERN32>(kp, X, a, order, n, cls, max_n, s);
        else launch_all<float, HM_MATERN32>(kp, X, a, order, n, cls, max_n, s);
    } else {
        aca_run_k1(f64, kp, X, a, order, n, cls, max_n, s);
    }
}

}  // namespace hm
