// hm_aca_team_f.cu -- the team ACA kernels (hm_aca_team.cuh) in float for the
// Gaussian and Matern-3/2 kernels, with the double ones in hm_aca_team_d.cu
// (separate units so that they compile in parallel).
#include "hm_aca_team.cuh"

namespace hm {

bool aca_team_gm_f(const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                   const uint32_t* order, int64_t n, int cls, int shape, int KT, cudaStream_t s)
{
    return kp.kernel == HM_GAUSSIAN
               ? launch_team_class<float, HM_GAUSSIAN>(kp, X, a, order, n, cls, shape, KT, s)
               : launch_team_class<float, HM_MATERN32>(kp, X, a, order, n, cls, shape, KT, s);
}

}  // namespace hm
