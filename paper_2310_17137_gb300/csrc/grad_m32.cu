// Fused MLL-gradient backward instances for one kernel family (see grad.cuh).
#include "grad.cuh"

namespace ap {
cudaError_t launch_grad_m32(const GradParams& p, int D, int C, cudaStream_t st) {
    return dispatch_grad<AP_MATERN32>(p, D, C, st);
}
}  // namespace ap
