// Cached block-Cholesky factors (Sec. 3, "Cached Cholesky Factors"; Table 6:
// (1/3) n b^2 flops, n b memory).
//
// For every diagonal block K_hat_II (b x b, the last one possibly short and
// padded with the identity to a whole number of 64 x 64 tiles):
//   1. build K_hat_II in FP64 directly from the FP32 inputs;
//   2. factor it in FP64 by a right-looking tiled Cholesky: POTRF of the
//      diagonal tile (which also inverts L_kk), TRSM of the panel below it as
//      a product with L_kk^{-T}, SYRK/GEMM update of the trailing tiles (FP64
//      FMA here, or exact integer slice products on the tensor cores in
//      ozaki.cu); all blocks of a group advance together, one launch per phase;
//   3. form the inverse factor L^{-1} tile by tile (diagonal tiles from the
//      FP64 tile inverses, off-diagonal tiles by the block recurrence
//      X_ik = -L_ii^{-1} sum_{j=k}^{i-1} L_ij X_jk) and store it packed in FP32.
// The per-step block solve Delta = L^{-T} (L^{-1} R_I) then becomes two
// parallel triangular products instead of two sequential substitutions.
#include <math.h>

#include "ap_internal.cuh"

namespace ap {
namespace {

constexpr int T = kTile;
constexpr int TP = kTile + 1;  // padded shared-memory row stride

__device__ __forceinline__ double phi_fp64(int kernel, double r2) {
    if (kernel == AP_RBF) return exp(-0.5 * r2);
    if (kernel == AP_MATERN32) {
        const double u = sqrt(3.0 * r2);
        return (1.0 + u) * exp(-u);
    }
    const double u = sqrt(5.0 * r2);
    return (1.0 + u + u * u / 3.0) * exp(-u);
}

// lower-triangular tile index t -> (i, j), j <= i
__device__ __forceinline__ void tri_index(int64_t t, int& i, int& j) {
    int ii = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while ((int64_t)ii * (ii + 1) / 2 > t) --ii;
    i = ii;
    j = (int)(t - (int64_t)ii * (ii + 1) / 2);
}

__device__ __forceinline__ int64_t packed_tile(int i, int k) { return (int64_t)i * (i + 1) / 2 + k; }

__global__ void __launch_bounds__(256) build_kii_kernel(const CacheParams cp, int64_t blk0, double* A) {
    const int z = blockIdx.y;
    const int64_t blk = blk0 + z;
    const int64_t ld = (int64_t)cp.nt * T;
    int ti, tj;
    tri_index(blockIdx.x, ti, tj);
    const int64_t lo = blk * cp.b;
    const int64_t bJ = min(cp.b, cp.n - lo);
    double* Ab = A + (int64_t)z * ld * ld;
    for (int t = threadIdx.x; t < T * T; t += blockDim.x) {
        const int r = t / T, q = t % T;
        const int64_t li = (int64_t)ti * T + r, lj = (int64_t)tj * T + q;
        double v;
        if (li < bJ && lj < bJ) {
            const float* xi = cp.X + (lo + li) * cp.d;
            const float* xj = cp.X + (lo + lj) * cp.d;
            double r2 = 0.0;
            for (int k = 0; k < cp.d; ++k) {
                const double df = ((double)xi[k] - (double)xj[k]) / cp.ell[k];
                r2 += df * df;
            }
            v = cp.s * phi_fp64(cp.kernel, r2);
            if (li == lj) v += cp.noise;
        } else {
            v = (li == lj) ? 1.0 : 0.0;
        }
        Ab[li * ld + lj] = v;
    }
}

// Factor the diagonal tile (k, k) in place and write its inverse to Dinv.
__global__ void __launch_bounds__(256) potrf_diag_kernel(double* A, int nt, int k, double* Dinv, int* bad) {
    extern __shared__ double pd_sm[];
    double* a = pd_sm;
    double* x = pd_sm + T * TP;
    __shared__ int s_bad;
    const int z = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    const int64_t ld = (int64_t)nt * T;
    double* Ab = A + (int64_t)z * ld * ld + (int64_t)k * T * ld + (int64_t)k * T;
    for (int t = tid; t < T * T; t += nth) {
        const int r = t / T, q = t % T;
        a[r * TP + q] = (q <= r) ? Ab[r * ld + q] : 0.0;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < T; ++j) {
        if (tid == 0) {
            double p = a[j * TP + j];
            if (!(p > 0.0) || !isfinite(p)) {
                s_bad = 1;
                p = 1.0;
            }
            a[j * TP + j] = sqrt(p);
        }
        __syncthreads();
        const double ljj = a[j * TP + j];
        for (int i = j + 1 + tid; i < T; i += nth) a[i * TP + j] /= ljj;
        __syncthreads();
        const int rem = T - j - 1;
        for (int t = tid; t < rem * rem; t += nth) {
            const int i = j + 1 + t / rem, l = j + 1 + t % rem;
            if (l <= i) a[i * TP + l] -= a[i * TP + j] * a[l * TP + j];
        }
        __syncthreads();
    }
    // inverse of the lower-triangular tile, one column per thread
    if (tid < T) {
        const int c = tid;
        for (int i = 0; i < c; ++i) x[i * TP + c] = 0.0;
        x[c * TP + c] = 1.0 / a[c * TP + c];
        for (int i = c + 1; i < T; ++i) {
            double s = 0.0;
            for (int q = c; q < i; ++q) s += a[i * TP + q] * x[q * TP + c];
            x[i * TP + c] = -s / a[i * TP + i];
        }
    }
    __syncthreads();
    double* Db = Dinv + ((int64_t)z * nt + k) * T * T;
    for (int t = tid; t < T * T; t += nth) {
        const int r = t / T, q = t % T;
        if (q <= r) Ab[r * ld + q] = a[r * TP + q];
        Db[t] = x[r * TP + q];
    }
    if (tid == 0 && s_bad) bad[z] = 1;
}

// A_ik <- A_ik L_kk^{-T} for the tiles i > k of the panel.
__global__ void __launch_bounds__(256) trsm_kernel(double* A, int nt, int k, const double* Dinv) {
    extern __shared__ double ts_sm[];
    double* sa = ts_sm;
    double* sd = ts_sm + T * TP;
    const int z = blockIdx.y, tid = threadIdx.x;
    const int i = k + 1 + blockIdx.x;
    const int64_t ld = (int64_t)nt * T;
    double* Aik = A + (int64_t)z * ld * ld + (int64_t)i * T * ld + (int64_t)k * T;
    const double* Db = Dinv + ((int64_t)z * nt + k) * T * T;
    for (int t = tid; t < T * T; t += 256) {
        const int r = t / T, q = t % T;
        sa[r * TP + q] = Aik[r * ld + q];
        sd[r * TP + q] = Db[t];
    }
    __syncthreads();
    const int tr = tid / 16, tc = tid % 16;
    double acc[4][4] = {};
    for (int p = 0; p < T; ++p) {
        double av[4], dv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) av[u] = sa[(tr + 16 * u) * TP + p];
#pragma unroll
        for (int v = 0; v < 4; ++v) dv[v] = sd[(tc + 16 * v) * TP + p];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], dv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) Aik[(int64_t)(tr + 16 * u) * ld + tc + 16 * v] = acc[u][v];
}

// A_ij -= A_ik A_jk^T for the trailing lower tiles k < j <= i.
__global__ void __launch_bounds__(256) syrk_kernel(double* A, int nt, int k) {
    extern __shared__ double sy_sm[];
    double* sa = sy_sm;
    double* sb = sy_sm + T * TP;
    const int z = blockIdx.y, tid = threadIdx.x;
    int ii, jj;
    tri_index(blockIdx.x, ii, jj);
    const int i = k + 1 + ii, j = k + 1 + jj;
    const int64_t ld = (int64_t)nt * T;
    double* Ab = A + (int64_t)z * ld * ld;
    const double* Aik = Ab + (int64_t)i * T * ld + (int64_t)k * T;
    const double* Ajk = Ab + (int64_t)j * T * ld + (int64_t)k * T;
    double* Aij = Ab + (int64_t)i * T * ld + (int64_t)j * T;
    for (int t = tid; t < T * T; t += 256) {
        const int r = t / T, q = t % T;
        sa[r * TP + q] = Aik[r * ld + q];
        sb[r * TP + q] = Ajk[r * ld + q];
    }
    __syncthreads();
    const int tr = tid / 16, tc = tid % 16;
    double acc[4][4] = {};
    for (int p = 0; p < T; ++p) {
        double av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) av[u] = sa[(tr + 16 * u) * TP + p];
#pragma unroll
        for (int v = 0; v < 4; ++v) bv[v] = sb[(tc + 16 * v) * TP + p];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            double* dst = Aij + (int64_t)(tr + 16 * u) * ld + tc + 16 * v;
            *dst -= acc[u][v];
        }
}

// Diagonal tiles of the packed FP32 inverse factor.
__global__ void __launch_bounds__(256) pack_diag_kernel(const double* Dinv, int nt, int64_t blk0,
                                                        int64_t ntri, float* Linv) {
    const int z = blockIdx.y, k = blockIdx.x;
    const double* Db = Dinv + ((int64_t)z * nt + k) * T * T;
    float* dst = Linv + ((blk0 + z) * ntri + packed_tile(k, k)) * T * T;
    for (int t = threadIdx.x; t < T * T; t += 256) dst[t] = (float)Db[t];
}

// Row of tiles i of L^{-1}: X_ik = -Dinv_ii * sum_{j=k}^{i-1} L_ij X_jk for k < i.
__global__ void __launch_bounds__(256) tri_inv_step_kernel(const double* A, const double* Dinv, int nt,
                                                           int i, int64_t blk0, int64_t ntri, float* Linv) {
    __shared__ float sl[T * TP];
    __shared__ float sx[T * TP];
    const int z = blockIdx.y, k = blockIdx.x, tid = threadIdx.x;
    const int64_t ld = (int64_t)nt * T;
    const double* Ab = A + (int64_t)z * ld * ld;
    float* Lb = Linv + (blk0 + z) * ntri * T * T;
    const int tr = tid / 16, tc = tid % 16;
    float acc[4][4] = {};
    for (int j = k; j < i; ++j) {
        __syncthreads();
        const double* Lij = Ab + (int64_t)i * T * ld + (int64_t)j * T;
        const float* Xjk = Lb + packed_tile(j, k) * T * T;
        for (int t = tid; t < T * T; t += 256) {
            const int r = t / T, q = t % T;
            sl[r * TP + q] = (float)Lij[r * ld + q];
            sx[r * TP + q] = Xjk[t];
        }
        __syncthreads();
        for (int p = 0; p < T; ++p) {
            float lv[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) lv[u] = sl[(tr + 16 * u) * TP + p];
#pragma unroll
            for (int v = 0; v < 4; ++v) xv[v] = sx[p * TP + tc + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(lv[u], xv[v], acc[u][v]);
        }
    }
    __syncthreads();
    const double* Db = Dinv + ((int64_t)z * nt + i) * T * T;
    for (int t = tid; t < T * T; t += 256) {
        const int r = t / T, q = t % T;
        sl[r * TP + q] = (float)Db[t];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) sx[(tr + 16 * u) * TP + tc + 16 * v] = acc[u][v];
    __syncthreads();
    float out[4][4] = {};
    for (int p = 0; p < T; ++p) {
        float dv[4], tv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) dv[u] = sl[(tr + 16 * u) * TP + p];
#pragma unroll
        for (int v = 0; v < 4; ++v) tv[v] = sx[p * TP + tc + 16 * v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) out[u][v] = fmaf(dv[u], tv[v], out[u][v]);
    }
    float* dst = Lb + packed_tile(i, k) * T * T;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[(tr + 16 * u) * T + tc + 16 * v] = -out[u][v];
}

}  // namespace

cudaError_t cache_factor_group(const CacheParams& cp, int64_t blk0, int g, double* A, double* Dinv,
                               float* Linv, int* bad, const OzWork* oz, cudaStream_t st, int64_t* launches) {
    const int nt = cp.nt;
    const int64_t ntri = (int64_t)nt * (nt + 1) / 2;
    const size_t smem2 = 2 * sizeof(double) * T * TP;
    cudaError_t err;
    if ((err = cudaFuncSetAttribute(potrf_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2)))
        return err;
    if ((err = cudaFuncSetAttribute(trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2)))
        return err;
    if ((err = cudaFuncSetAttribute(syrk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2)))
        return err;
    int64_t nl = 0;
    build_kii_kernel<<<dim3((unsigned)ntri, g), 256, 0, st>>>(cp, blk0, A);
    ++nl;
    for (int k = 0; k < nt; ++k) {
        potrf_diag_kernel<<<g, 256, smem2, st>>>(A, nt, k, Dinv, bad);
        ++nl;
        if (k + 1 < nt) {
            const int rem = nt - k - 1;
            trsm_kernel<<<dim3(rem, g), 256, smem2, st>>>(A, nt, k, Dinv);
            ++nl;
            if (oz) {
                if ((err = launch_oz_update(A, nt, k, g, oz->S, oz->E, oz->err, st, &nl)) != cudaSuccess) return err;
            } else {
                syrk_kernel<<<dim3((unsigned)((int64_t)rem * (rem + 1) / 2), g), 256, smem2, st>>>(A, nt, k);
                ++nl;
            }
        }
    }
    pack_diag_kernel<<<dim3(nt, g), 256, 0, st>>>(Dinv, nt, blk0, ntri, Linv);
    ++nl;
    for (int i = 1; i < nt; ++i) {
        tri_inv_step_kernel<<<dim3(i, g), 256, 0, st>>>(A, Dinv, nt, i, blk0, ntri, Linv);
        ++nl;
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
}

}  // namespace ap
