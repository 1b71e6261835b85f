// ap_sfu_rates: measured throughput of the two SFU operations the kernel
// evaluation is made of (exp2 for every kernel, sqrt for the Matern kernels),
// in results per SM clock.  One CTA of 1024 threads per SM (the dynamic shared
// memory request keeps a second CTA off the SM) runs eight independent chains
// per thread; each CTA times its own loop with the SM cycle counter, so the
// rate does not depend on the clock the GPU happens to run at.  No counterpart
// in the paper: the benchmark divides by these rates to place the tensor-core
// residual update on its roofline.
#include <algorithm>
#include <vector>

#include "kmv_fp32.cuh"

namespace ap {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeChains = 8;
constexpr int kProbeIters = 2048;
constexpr size_t kProbeSmem = 120 * 1024;

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) sfu_probe_kernel(float* sink, long long* cycles) {
    float x[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) x[j] = 0.5f + 0.01f * j + 1e-6f * threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) {
            // ex2(-x) keeps x in (0.5, 1); sqrt keeps it in (0, 1]
            if (OP == 0) x[j] = ex2_approx(-x[j]);
            else x[j] = sqrt_approx(x[j]);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) s += x[j];
    sink[blockIdx.x * kProbeThreads + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
cudaError_t probe(int sms, float* sink, long long* cycles_dev, double* rate) {
    auto fn = sfu_probe_kernel<OP>;
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeSmem);
    if (err != cudaSuccess) return err;
    std::vector<long long> cyc((size_t)sms);
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
        fn<<<sms, kProbeThreads, kProbeSmem>>>(sink, cycles_dev);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if ((err = cudaMemcpy(cyc.data(), cycles_dev, sizeof(long long) * sms, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return err;
    }
    std::sort(cyc.begin(), cyc.end());
    const double median = (double)cyc[cyc.size() / 2];
    *rate = median > 0 ? (double)kProbeThreads * kProbeChains * kProbeIters / median : 0.0;
    return cudaSuccess;
}

}  // namespace
}  // namespace ap

extern "C" ap_status ap_sfu_rates(double* ex2_per_clk_sm, double* sqrt_per_clk_sm) {
    using namespace ap;
    if (!ex2_per_clk_sm || !sqrt_per_clk_sm) return AP_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return AP_ERR_CUDA;
    }
    float* sink = nullptr;
    long long* cycles = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * sms * kProbeThreads) != cudaSuccess ||
        cudaMalloc(&cycles, sizeof(long long) * sms) != cudaSuccess) {
        cudaFree(sink);
        cudaGetLastError();
        return AP_ERR_NOMEM;
    }
    cudaError_t err = probe<0>(sms, sink, cycles, ex2_per_clk_sm);
    if (err == cudaSuccess) err = probe<1>(sms, sink, cycles, sqrt_per_clk_sm);
    cudaFree(sink);
    cudaFree(cycles);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return AP_ERR_CUDA;
    }
    return AP_OK;
}
