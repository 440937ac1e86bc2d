// hm_aca_team_d.cu -- the team ACA kernels (hm_aca_team.cuh) in double for the
// Gaussian and Matern-3/2 kernels, and the dispatch of both precisions.
#include "hm_aca_team.cuh"

namespace hm {

bool aca_team_gm_f(const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                   const uint32_t* order, int64_t n, int cls, int shape, int KT, cudaStream_t s);

bool aca_team_gm(bool f64, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                 const uint32_t* order, int64_t n, int cls, int shape, int KT, cudaStream_t s)
{
    if (!f64) return aca_team_gm_f(kp, X, a, order, n, cls, shape, KT, s);
    return kp.kernel == HM_GAUSSIAN
               ? launch_team_class<double, HM_GAUSSIAN>(kp, X, a, order, n, cls, shape, KT, s)
               : launch_team_class<double, HM_MATERN32>(kp, X, a, order, n, cls, shape, KT, s);
}

}  // namespace hm
