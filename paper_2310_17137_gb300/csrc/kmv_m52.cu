// FP32 kernel-matrix product instances for one kernel family (see kmv_fp32.cuh).
#include "kmv_fp32.cuh"

namespace ap {
cudaError_t launch_kmv_m52(const KmvParams& p, int D, int C, cudaStream_t st) {
    return dispatch_kmv<AP_MATERN52>(p, D, C, st);
}
}  // namespace ap
