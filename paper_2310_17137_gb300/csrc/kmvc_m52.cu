// Compensated kernel-matrix product instances for one kernel family (see kmv_comp.cuh).
#include "kmv_comp.cuh"

namespace ap {
cudaError_t launch_kmv_comp_m52(const KmvParams& p, int D, int C, cudaStream_t st) {
    return dispatch_kmv_comp<AP_MATERN52>(p, D, C, st);
}
}  // namespace ap
