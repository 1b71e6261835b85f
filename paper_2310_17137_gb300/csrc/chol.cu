// Cached block-Cholesky factors (Sec. 3, "Cached Cholesky Factors"; Table 6:
// (1/3) n b^2 flops, n b memory).
//
// For every diagonal block K_hat_II (b x b, the last one possibly short and
// padded with the identity to a whole number of 64 x 64 tiles):
//   1. build K_hat_II in FP64 directly from the FP32 inputs;
//   2. factor it in FP64 by a right-looking tiled Cholesky: POTRF of the
//      diagonal tile (which also inverts L_kk), TRSM of the panel below it as
//      a product with L_kk^{-T}, SYRK/GEMM update of the trailing tiles (the
//      products as FP64 FMAs here, or as exact integer slice products on the
//      tensor cores in ozaki.cu); all blocks of a group advance together, one
//      launch per phase;
//   3. form the inverse factor L^{-1} tile by tile (diagonal tiles from the
//      FP64 tile inverses, off-diagonal tiles by the block recurrence
//      X_ik = -L_ii^{-1} sum_{j=k}^{i-1} L_ij X_jk) and store it packed in FP32.
// The per-step block solve Delta = L^{-T} (L^{-1} R_I) then becomes two
// parallel triangular products instead of two sequential substitutions.
#include <math.h>

#include <algorithm>

#include "ap_internal.cuh"

namespace ap {
namespace {

constexpr int T = kTile;
constexpr int TP = kTile + 1;  // padded shared-memory row stride

// ---------------------------------------------------------------- FP64 phi
// The kernel profile phi(r^2) in FP64 for K_II, built from a handful of FP64
// FMAs instead of the library exp and sqrt (FP64 arithmetic is scarce on this
// part; the library calls cost ~90 FP64 operations per entry).
//
// exp(x), x <= 0: Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989): x = (64 k + j) ln2/64 + r with
// |r| <= ln2/128, e^x = 2^k 2^(j/64) e^r.  ln2/64 is split into the double
// nearest to it and the double nearest to the remainder, so r is exact to a
// rounding; e^r - 1 is its Taylor polynomial to degree 6 (truncation below
// r^7/7! < 2^-62 relative).  2^k is assembled from its exponent bits.  Below
// x = -708 the result is 0 (e^-708 ~ 3e-308, far below any kernel value
// that matters next to sigma^2).
// sqrt(x): the FP32 reciprocal square root (relative error < 2^-22), one
// Newton step for 1/sqrt(x) in FP64 (error ~1.5 e^2 < 2^-44), then one
// Newton correction of s = x y (error ~e^2, below the last bit).
constexpr double kLn2By64Hi = 0x1.62e42fefa39efp-7;   // double nearest to ln2 / 64
constexpr double kLn2By64Lo = 0x1.abc9e3b39803fp-62;  // ln2 / 64 - kLn2By64Hi, rounded
constexpr double k64ByLn2 = 92.33248261689366;        // 64 / ln2

__device__ __forceinline__ double exp_nonpos(double x, const double* tab2) {
    if (!(x >= -708.0)) return 0.0;  // also maps NaN to 0; callers pass finite x
    const double nf = rint(x * k64ByLn2);
    const int n = (int)nf;
    const double r = fma(-nf, kLn2By64Lo, fma(-nf, kLn2By64Hi, x));
    double q = 1.0 / 720.0;
    q = fma(q, r, 1.0 / 120.0);
    q = fma(q, r, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    q = fma(q, r, 1.0);
    const double t = tab2[n & 63];
    const double y = fma(t, q * r, t);
    const int k = n >> 6;  // floor(n / 64), in [-1022, 0]
    return y * __longlong_as_double((long long)(k + 1023) << 52);
}

__device__ __forceinline__ double sqrt_nonneg(double x) {
    if (x < 1e-36) return 0.0;  // phi is flat at 0: the error is below the last bit
    if (x > 1e12) return 1e6;   // e^-sqrt(x) underflows either way
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)x));
    double y = (double)yf;
    y = fma(0.5 * y, fma(-x * y, y, 1.0), y);
    const double s = x * y;
    return fma(0.5 * y, fma(-s, s, x), s);
}

__device__ __forceinline__ double phi_fp64(int kernel, double r2, const double* tab2) {
    if (kernel == AP_RBF) return exp_nonpos(-0.5 * r2, tab2);
    if (kernel == AP_MATERN32) {
        const double u = sqrt_nonneg(3.0 * r2);
        return (1.0 + u) * exp_nonpos(-u, tab2);
    }
    const double u = sqrt_nonneg(5.0 * r2);
    return fma(u, fma(u, 1.0 / 3.0, 1.0), 1.0) * exp_nonpos(-u, tab2);
}

// 2^(j/64), j = 0..63, into shared memory (first 64 threads; caller syncs)
__device__ __forceinline__ void fill_exp2_table(double* tab2) {
    if (threadIdx.x < 64) tab2[threadIdx.x] = exp2((double)threadIdx.x / 64.0);
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
    __shared__ double s_tab[64];
    __shared__ double s_inv_ell[AP_MAX_DIM];
    __shared__ double s_xi[AP_MAX_DIM * T], s_xj[AP_MAX_DIM * T];  // dimension-major
    const int z = blockIdx.y;
    const int64_t blk = blk0 + z;
    const int64_t ld = (int64_t)cp.nt * T;
    const int d = cp.d;
    int ti, tj;
    tri_index(blockIdx.x, ti, tj);
    const int64_t lo = blk * cp.b;
    const int64_t bJ = min(cp.b, cp.n - lo);
    double* Ab = A + (int64_t)z * ld * ld;
    fill_exp2_table(s_tab);
    if (threadIdx.x < d) s_inv_ell[threadIdx.x] = 1.0 / cp.ell[threadIdx.x];
    // the tile's row and column points (rows past the block are never read)
    for (int t = threadIdx.x; t < T * d; t += blockDim.x) {
        const int r = t / d, k = t % d;
        const int64_t li = (int64_t)ti * T + r, lj = (int64_t)tj * T + r;
        s_xi[k * T + r] = li < bJ ? (double)cp.X[(lo + li) * d + k] : 0.0;
        s_xj[k * T + r] = lj < bJ ? (double)cp.X[(lo + lj) * d + k] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T * T; t += blockDim.x) {
        const int r = t / T, q = t % T;
        const int64_t li = (int64_t)ti * T + r, lj = (int64_t)tj * T + q;
        double v;
        if (li < bJ && lj < bJ) {
            // the difference of two FP32 values is exact in FP64
            double r2 = 0.0;
            for (int k = 0; k < d; ++k) {
                const double df = (s_xi[k * T + r] - s_xj[k * T + q]) * s_inv_ell[k];
                r2 = fma(df, df, r2);
            }
            v = cp.s * phi_fp64(cp.kernel, r2, s_tab);
            if (li == lj) v += cp.noise;
        } else {
            v = (li == lj) ? 1.0 : 0.0;
        }
        Ab[li * ld + lj] = v;
    }
}

// FP64 phi at given squared distances (verification of the cache's kernel values)
__global__ void __launch_bounds__(256) phi_fp64_eval_kernel(int kernel, const double* r2, int64_t count,
                                                            double* out) {
    __shared__ double s_tab[64];
    fill_exp2_table(s_tab);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = phi_fp64(kernel, r2[i], s_tab);
}

// Factor the diagonal tile (k, k) in place and write its inverse to Dinv.
// 1/sqrt(p) for a pivot: the FP32 reciprocal square root refined by two
// Newton steps in FP64 (relative error 2^-22 -> 2^-44 -> below the last bit);
// outside the FP32 range the library square root and division.
__device__ __forceinline__ double rsqrt_pivot(double p) {
    if (!(p > 1e-30 && p < 1e30)) return 1.0 / sqrt(p);
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)p));
    double y = (double)yf;
    y = fma(0.5 * y, fma(-p * y, y, 1.0), y);
    return fma(0.5 * y, fma(-p * y, y, 1.0), y);
}

__global__ void __launch_bounds__(256) potrf_diag_kernel(double* A, int nt, int k, double* Dinv, int* bad) {
    extern __shared__ double pd_sm[];
    double* a = pd_sm;
    double* x = pd_sm + T * TP;
    __shared__ double s_rd[T];  // 1 / L_jj
    __shared__ int s_bad;
    const int z = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
    const int ty = tid / 16, tx = tid % 16;
    const int64_t ld = (int64_t)nt * T;
    double* Ab = A + (int64_t)z * ld * ld + (int64_t)k * T * ld + (int64_t)k * T;
    for (int t = tid; t < T * T; t += nth) {
        const int r = t / T, q = t % T;
        a[r * TP + q] = (q <= r) ? Ab[r * ld + q] : 0.0;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < T; ++j) {
        // every thread derives the pivot's reciprocal square root itself
        double pv = a[j * TP + j];
        const bool badp = !(pv > 0.0) || !isfinite(pv);
        if (badp) pv = 1.0;
        const double rj = rsqrt_pivot(pv);
        __syncthreads();  // everyone has read the pivot
        if (tid == 0) {
            if (badp) s_bad = 1;
            const double l = pv * rj;
            a[j * TP + j] = fma(0.5 * rj, fma(-l, l, pv), l);  // sqrt(pv), Newton-corrected
            s_rd[j] = rj;
        }
        for (int i = j + 1 + tid; i < T; i += nth) a[i * TP + j] *= rj;
        __syncthreads();
        // trailing update of the lower triangle, rows j+1+ty+16a, columns j+1+tx+16b
        for (int i = j + 1 + ty; i < T; i += 16) {
            const double aij = a[i * TP + j];
            for (int l = j + 1 + tx; l <= i; l += 16) a[i * TP + l] = fma(-aij, a[l * TP + j], a[i * TP + l]);
        }
        __syncthreads();
    }
    // inverse of the lower-triangular tile, one column per thread, the inner
    // products in four independent partial sums
    if (tid < T) {
        const int c = tid;
        for (int i = 0; i < c; ++i) x[i * TP + c] = 0.0;
        x[c * TP + c] = s_rd[c];
        for (int i = c + 1; i < T; ++i) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int q = c;
            for (; q + 3 < i; q += 4) {
                s0 = fma(a[i * TP + q], x[q * TP + c], s0);
                s1 = fma(a[i * TP + q + 1], x[(q + 1) * TP + c], s1);
                s2 = fma(a[i * TP + q + 2], x[(q + 2) * TP + c], s2);
                s3 = fma(a[i * TP + q + 3], x[(q + 3) * TP + c], s3);
            }
            for (; q < i; ++q) s0 = fma(a[i * TP + q], x[q * TP + c], s0);
            x[i * TP + c] = -((s0 + s1) + (s2 + s3)) * s_rd[i];
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

// FP32 copies of the off-diagonal factor tiles L_ij (i > j) for the inverse
// recurrence, converted once and kept in the unused upper triangle of the FP64
// workspace: L_ij as a row-major 64 x 64 float tile in the first half of the
// rows of tile (j, i).
__device__ __forceinline__ float* lf32_tile(double* Ab, int64_t ld, int i, int j) {
    return reinterpret_cast<float*>(Ab + (int64_t)j * T * ld + (int64_t)i * T);
}

__global__ void __launch_bounds__(256) lower_to_f32_kernel(double* A, int nt) {
    const int z = blockIdx.y;
    int i, j;
    tri_index(blockIdx.x, i, j);  // i >= j; the diagonal tiles are not needed
    if (i == j) return;
    const int64_t ld = (int64_t)nt * T;
    double* Ab = A + (int64_t)z * ld * ld;
    const double* src = Ab + (int64_t)i * T * ld + (int64_t)j * T;
    float* dst = lf32_tile(Ab, ld, i, j);
    for (int t = threadIdx.x; t < T * T; t += 256) {
        const int r = t / T, q = t % T;
        dst[(int64_t)r * 2 * ld + q] = (float)src[(int64_t)r * ld + q];
    }
}

// Row of tiles i of L^{-1}: X_ik = -X_ii * sum_{j=k}^{i-1} L_ij X_jk for k < i
// (X_ii = L_ii^{-1} is already packed).  Thread (tr, tc) owns rows 4 tr .. + 3
// and columns 4 tc .. + 3 of the tile; L is staged transposed and X row-major,
// so every K step is two 16-byte shared loads for 16 FMAs.
constexpr int TQ = T + 4;  // padded stride: rows stay 16-byte aligned, transposed stores spread over banks

__global__ void __launch_bounds__(256) tri_inv_step_kernel(double* A, int nt, int i, int64_t blk0, int64_t ntri,
                                                           float* Linv) {
    __shared__ __align__(16) float slt[T * TQ];  // slt[p][r] = L_ij(r, p)
    __shared__ __align__(16) float sx[T * TQ];   // sx[p][c]  = X_jk(p, c)
    const int z = blockIdx.y, k = blockIdx.x, tid = threadIdx.x;
    const int64_t ld = (int64_t)nt * T;
    double* Ab = A + (int64_t)z * ld * ld;
    float* Lb = Linv + (blk0 + z) * ntri * T * T;
    const int tr = tid / 16, tc = tid % 16;
    float acc[4][4] = {};
    auto kstep_product = [&]() {
#pragma unroll 8
        for (int p = 0; p < T; ++p) {
            const float4 lv = *reinterpret_cast<const float4*>(&slt[p * TQ + 4 * tr]);
            const float4 xv = *reinterpret_cast<const float4*>(&sx[p * TQ + 4 * tc]);
            const float l4[4] = {lv.x, lv.y, lv.z, lv.w}, x4[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(l4[u], x4[v], acc[u][v]);
        }
    };
    for (int j = k; j < i; ++j) {
        __syncthreads();
        const float* Lij = lf32_tile(Ab, ld, i, j);
        const float* Xjk = Lb + packed_tile(j, k) * T * T;
        for (int t = tid; t < T * T; t += 256) {
            const int r = t / T, q = t % T;
            slt[q * TQ + r] = Lij[(int64_t)r * 2 * ld + q];
            sx[r * TQ + q] = Xjk[t];
        }
        __syncthreads();
        kstep_product();
    }
    __syncthreads();
    // out = X_ii acc: X_ii staged transposed like L, acc row-major like X
    const float* Xii = Lb + packed_tile(i, i) * T * T;
    for (int t = tid; t < T * T; t += 256) {
        const int r = t / T, q = t % T;
        slt[q * TQ + r] = Xii[t];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        *reinterpret_cast<float4*>(&sx[(4 * tr + u) * TQ + 4 * tc]) =
            make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
    __syncthreads();
    kstep_product();
    float* dst = Lb + packed_tile(i, k) * T * T;
#pragma unroll
    for (int u = 0; u < 4; ++u)
        *reinterpret_cast<float4*>(&dst[(4 * tr + u) * T + 4 * tc]) =
            make_float4(-acc[u][0], -acc[u][1], -acc[u][2], -acc[u][3]);
}

}  // namespace

cudaError_t launch_phi_fp64_eval(int kernel, const double* r2, int64_t count, double* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
    phi_fp64_eval_kernel<<<(unsigned)blocks, 256, 0, st>>>(kernel, r2, count, out);
    return cudaGetLastError();
}

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
            if (oz) {
                if ((err = launch_oz_trsm(A, Dinv, nt, k, g, oz->S, oz->E, oz->err, st, &nl)) != cudaSuccess)
                    return err;
                if ((err = launch_oz_update(A, nt, k, g, oz->S, oz->E, oz->err, st, &nl)) != cudaSuccess) return err;
            } else {
                trsm_kernel<<<dim3(rem, g), 256, smem2, st>>>(A, nt, k, Dinv);
                ++nl;
                syrk_kernel<<<dim3((unsigned)((int64_t)rem * (rem + 1) / 2), g), 256, smem2, st>>>(A, nt, k);
                ++nl;
            }
        }
    }
    pack_diag_kernel<<<dim3(nt, g), 256, 0, st>>>(Dinv, nt, blk0, ntri, Linv);
    ++nl;
    lower_to_f32_kernel<<<dim3((unsigned)ntri, g), 256, 0, st>>>(A, nt);
    ++nl;
    for (int i = 1; i < nt; ++i) {
        tri_inv_step_kernel<<<dim3(i, g), 256, 0, st>>>(A, nt, i, blk0, ntri, Linv);
        ++nl;
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
}

}  // namespace ap
