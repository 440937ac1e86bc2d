// hm_aca_team_k1.cu -- the team ACA kernels (hm_aca_team.cuh) for the Matern
// kernel of order 1, both precisions.
#include "hm_aca_team.cuh"

namespace hm {

bool aca_team_k1(bool f64, const KernelParams& kp, const DeviceCoords& X, const AcaArgs& a,
                 const uint32_t* order, int64_t n, int cls, int shape, int KT, cudaStream_t s)
{
    return f64 ? launch_team_class<double, HM_MATERN_K1>(kp, X, a, order, n, cls, shape, KT, s)
               : launch_team_class<float, HM_MATERN_K1>(kp, X, a, order, n, cls, shape, KT, s);
}

}  // namespace hm
