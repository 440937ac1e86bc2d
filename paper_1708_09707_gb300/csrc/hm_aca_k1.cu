// hm_aca_k1.cu -- batched ACA (Alg. 2, Sec. 5.4.1) for the Matern kernel of
// order 1 (Sec. 6.2): the cluster kernels here, the team kernels in
// hm_aca_team_k1.cu (units of their own so that they compile in parallel).
#include "hm_aca_impl.cuh"

namespace hm {

void aca_run_k1(bool f64, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                const uint32_t* order, int64_t n, int cls, int, int64_t max_n, cudaStream_t s)
{
    if (f64) launch_all<double, HM_MATERN_K1>(kp, X, a, order, n, cls, max_n, s);
    else launch_all<float, HM_MATERN_K1>(kp, X, a, order, n, cls, max_n, s);
}

}  // namespace hm
