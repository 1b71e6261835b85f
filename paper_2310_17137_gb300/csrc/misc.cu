// Input preparation, padding copies, the stand-alone norm/selection pass and
// the kernel-family dispatch of the FP32 product.
#include <math.h>

#include "kmv_fp32.cuh"

namespace ap {

double kernel_input_scale(int kernel) {
    if (kernel == AP_RBF) return sqrt(0.5 * 1.4426950408889634);  // sqrt(log2(e) / 2)
    if (kernel == AP_MATERN32) return sqrt(3.0);
    return sqrt(5.0);
}

int kmv_rows_per_cta(int D, int C) { return kKmvThreads * rows_per_thread(D, C); }

cudaError_t launch_kmv(int kernel, const KmvParams& p, int D, int C, cudaStream_t st) {
    switch (kernel) {
        case AP_RBF: return launch_kmv_rbf(p, D, C, st);
        case AP_MATERN32: return launch_kmv_m32(p, D, C, st);
        case AP_MATERN52: return launch_kmv_m52(p, D, C, st);
        default: return cudaErrorInvalidValue;
    }
}

namespace {

struct ScaleVec {
    float v[AP_MAX_DIM];
};

// Xs[i, k] = fl(X[i, k] * sc_k) for k < d, 0 for the padding k in [d, D);
// sc_k = hi_k + lo_k, and Xs_lo gets X * sc_k - Xs (TwoProd remainder plus
// the lo part of the scale) when requested.  A NaN or Inf input sets *bad.
__global__ void prep_inputs_kernel(const float* __restrict__ X, int64_t n, int d, int D, const ScaleVec sh,
                                   const ScaleVec sl, float* __restrict__ Xs, float* __restrict__ Xs_lo,
                                   int* __restrict__ bad) {
    const int64_t total = n * D;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / D;
        const int k = (int)(t % D);
        float hi = 0.0f, lo = 0.0f;
        if (k < d && AP_CHK(i < n)) {
            const float x = X[i * d + k];
            if (!isfinite(x) && bad) *bad = 1;
            hi = x * sh.v[k];
            lo = fmaf(x, sh.v[k], -hi) + x * sl.v[k];
        }
        Xs[t] = hi;
        if (Xs_lo) Xs_lo[t] = lo;
    }
}

__global__ void pad_copy_kernel(const float* __restrict__ src, int64_t n, int c, float* __restrict__ dst, int C) {
    const int64_t total = n * C;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / C;
        const int k = (int)(t % C);
        dst[t] = k < c ? src[i * c + k] : 0.0f;
    }
}

__global__ void unpad_copy_kernel(const float* __restrict__ src, int64_t n, int C, float* __restrict__ dst, int c) {
    const int64_t total = n * c;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / c;
        const int k = (int)(t % c);
        dst[t] = src[i * C + k];
    }
}

unsigned grid_for(int64_t total) {
    int64_t g = (total + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

cudaError_t launch_prep_inputs(const float* X, int64_t n, int d, int D, const float* sc_hi, const float* sc_lo,
                               float* Xs, float* Xs_lo, int* bad, cudaStream_t st) {
    ScaleVec sh = {}, sl = {};
    for (int k = 0; k < d && k < AP_MAX_DIM; ++k) {
        sh.v[k] = sc_hi[k];
        sl.v[k] = sc_lo ? sc_lo[k] : 0.0f;
    }
    prep_inputs_kernel<<<grid_for(n * D), 256, 0, st>>>(X, n, d, D, sh, sl, Xs, Xs_lo, bad);
    return cudaGetLastError();
}

cudaError_t launch_pad_copy(const float* src, int64_t n, int c, float* dst, int C, cudaStream_t st) {
    pad_copy_kernel<<<grid_for(n * C), 256, 0, st>>>(src, n, c, dst, C);
    return cudaGetLastError();
}

cudaError_t launch_unpad_copy(const float* src, int64_t n, int C, float* dst, int c, cudaStream_t st) {
    unpad_copy_kernel<<<grid_for(n * c), 256, 0, st>>>(src, n, C, dst, c);
    return cudaGetLastError();
}

cudaError_t launch_norms_select(const float* R, int64_t n, int C, const EpiParams& e, int64_t tile_rows,
                                cudaStream_t st) {
    const dim3 grid((unsigned)e.ntiles, 1, 1);
    switch (C) {
        case 1: norms_select_kernel<1><<<grid, kKmvThreads, 0, st>>>(R, n, e, tile_rows); break;
        case 4: norms_select_kernel<4><<<grid, kKmvThreads, 0, st>>>(R, n, e, tile_rows); break;
        case 16: norms_select_kernel<16><<<grid, kKmvThreads, 0, st>>>(R, n, e, tile_rows); break;
        case 32: norms_select_kernel<32><<<grid, kKmvThreads, 0, st>>>(R, n, e, tile_rows); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ap

namespace ap {

int grad_rows_per_cta(int D, int C) { return 128 * ((D + C <= 40) ? 2 : 1); }

cudaError_t launch_kmv_comp(int kernel, const KmvParams& p, int D, int C, cudaStream_t st) {
    switch (kernel) {
        case AP_RBF: return launch_kmv_comp_rbf(p, D, C, st);
        case AP_MATERN32: return launch_kmv_comp_m32(p, D, C, st);
        case AP_MATERN52: return launch_kmv_comp_m52(p, D, C, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_grad(int kernel, const GradParams& p, int D, int C, cudaStream_t st) {
    switch (kernel) {
        case AP_RBF: return launch_grad_rbf(p, D, C, st);
        case AP_MATERN32: return launch_grad_m32(p, D, C, st);
        case AP_MATERN52: return launch_grad_m52(p, D, C, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ap

namespace ap {
namespace {

__device__ __forceinline__ float rademacher_at(uint64_t seed, uint64_t idx) {
    return (splitmix64_at(seed, idx) >> 63) ? 1.0f : -1.0f;
}

// B = [y - mu, z_1..z_l] (n x c); Z == nullptr draws z from SplitMix64(seed).
__global__ void assemble_rhs_kernel(const float* __restrict__ y, float mu, const float* __restrict__ Z, int l,
                                    uint64_t seed, int64_t n, float* __restrict__ B, float* __restrict__ Zout) {
    const int c = l + 1;
    const int64_t total = n * c;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / c;
        const int k = (int)(t % c);
        float v;
        if (k == 0) {
            v = y[i] - mu;
        } else {
            const int64_t zi = i * l + (k - 1);
            v = Z ? Z[zi] : rademacher_at(seed, (uint64_t)zi);
            if (Zout) Zout[zi] = v;
        }
        B[t] = v;
    }
}

// V = [u, z_1..z_l] from the solved W (n x C, column 0 = u) and B (n x c).
__global__ void assemble_v_kernel(const float* __restrict__ W, int C, const float* __restrict__ B, int c, int64_t n,
                                  float* __restrict__ V) {
    const int64_t total = n * C;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / C;
        const int k = (int)(t % C);
        V[t] = k == 0 ? W[i * C] : (k < c ? B[i * c + k] : 0.0f);
    }
}

// out[0] = sum_i W[i * C] * (Y ? Y[i * cy] : 1) in FP64 (the ticketed last CTA
// adds the per-CTA partials in order).
__global__ void dot0_kernel(const float* __restrict__ W, int C, const float* __restrict__ Y, int cy, int64_t n,
                            double* part, unsigned* ticket, double* out) {
    __shared__ double red[32];
    __shared__ int s_last;
    double v = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v += (double)W[i * C] * (Y ? (double)Y[i * cy] : 1.0);
    double t = cta_sum_d(v, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1u) ? 1 : 0;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double acc = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) acc += __ldcg(part + b);
        *out = acc;
        *ticket = 0u;
    }
}

}  // namespace

cudaError_t launch_assemble_rhs(const float* y, float mu, const float* Z, int l, uint64_t seed, int64_t n, float* B,
                                float* Zout, cudaStream_t st) {
    assemble_rhs_kernel<<<grid_for(n * (l + 1)), 256, 0, st>>>(y, mu, Z, l, seed, n, B, Zout);
    return cudaGetLastError();
}

cudaError_t launch_assemble_v(const float* W, int C, const float* B, int c, int64_t n, float* V, cudaStream_t st) {
    assemble_v_kernel<<<grid_for(n * C), 256, 0, st>>>(W, C, B, c, n, V);
    return cudaGetLastError();
}

constexpr unsigned kColsumGrid = 256;

cudaError_t launch_dot0(const float* W, int C, const float* Y, int cy, int64_t n, double* part, unsigned* ticket,
                       double* out, cudaStream_t st) {
    dot0_kernel<<<kColsumGrid, kKmvThreads, 0, st>>>(W, C, Y, cy, n, part, ticket, out);
    return cudaGetLastError();
}

}  // namespace ap

// ---------------------------------------------------- bounds-check self-test
namespace ap {
namespace {

// One thread reads element `index` of an 8-element buffer through AP_CHK: in
// the checked build an index outside [0, 8) is recorded and the read skipped.
__global__ void bounds_selftest_kernel(const float* __restrict__ buf, int index, float* __restrict__ out) {
    float v = 0.0f;
    if (AP_CHK(index >= 0 && index < 8)) v = buf[index];
    *out = v;
}

}  // namespace
}  // namespace ap

extern "C" ap_status ap_bounds_selftest(int32_t index) {
#ifdef AP_CHECKED
    float* d = nullptr;
    if (cudaMalloc(&d, 9 * sizeof(float)) != cudaSuccess) return AP_ERR_NOMEM;
    cudaMemset(d, 0, 9 * sizeof(float));
    ap::bounds_selftest_kernel<<<1, 1>>>(d, index, d + 8);
    const cudaError_t err = cudaDeviceSynchronize();
    cudaFree(d);
    return err == cudaSuccess ? AP_OK : AP_ERR_CUDA;
#else
    (void)index;
    return AP_ERR_UNSUPPORTED;
#endif
}
