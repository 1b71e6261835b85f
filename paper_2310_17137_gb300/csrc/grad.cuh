// Fused backward pass of the stochastic MLL gradient (Eq. loss_grad_unbiased):
// one sweep over all n^2 kernel entries that forms G_ij = sum_c alpha_c U_ic V_jc
// on the fly and contracts it with every derivative dK_ij / dtheta at once
// (d lengthscales, outputscale, noise).  No kernel block or G block is stored.
//
// With the pre-scaled inputs xs of the FP32 product (xs = c_K x / l, see
// kernel_input_scale) and t = |xs_i - xs_j|^2:
//   RBF  phi = 2^-t,                     psi = phi
//   M32  u = sqrt(t), phi = (1+u) e^-u,  psi = e^-u
//   M52  u = sqrt(t), phi = (1+u+u^2/3) e^-u, psi = (1+u) e^-u
// and dK/dl_k = s * kappa_K / (c_K^2 l_k) * psi * (xs_ik - xs_jk)^2 with
// kappa_K / c_K^2 = 2/log2(e), 1, 1/3; the host applies those factors.
#pragma once

#include "kmv_fp32.cuh"

namespace ap {

template <int KERN>
__device__ __forceinline__ void phi_psi_fp32(float t, float& phi, float& psi) {
    if constexpr (KERN == AP_RBF) {
        phi = ex2_approx(-t);
        psi = phi;
    } else if constexpr (KERN == AP_MATERN32) {
        const float u = sqrt_approx(t);
        const float e = ex2_approx(-u * kLog2e);
        phi = (1.0f + u) * e;
        psi = e;
    } else {
        const float u = sqrt_approx(t);
        const float e = ex2_approx(-u * kLog2e);
        psi = (1.0f + u) * e;
        phi = fmaf(u * u, (1.0f / 3.0f) * e, psi);
    }
}

constexpr int kGradThreads = 128;
constexpr int kGradTN = 64;

template <int D, int C>
struct GradShape {
    static constexpr int RM = (D + C <= 40) ? 2 : 1;
    static constexpr int ROWS = kGradThreads * RM;
};

template <int KERN, int D, int C>
__global__ void __launch_bounds__(kGradThreads) grad_kernel(const GradParams p) {
    constexpr int RM = GradShape<D, C>::RM;
    constexpr int ROWS = GradShape<D, C>::ROWS;
    constexpr int NA = D + 2;
    __shared__ __align__(16) float s_xb[kGradTN * D];
    __shared__ __align__(16) float s_v[kGradTN * C];
    __shared__ double red_d[32];
    __shared__ double s_tot[NA];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int S = gridDim.y, rank = blockIdx.y;
    const int64_t r0 = (int64_t)blockIdx.x * ROWS;
    const int64_t cs = ((p.n + S - 1) / S + kGradTN - 1) / kGradTN * kGradTN;
    const int64_t c_lo = rank * cs, c_hi = min(p.n, c_lo + cs);

    float xa[RM][D], ua[RM][C];
    double diag = 0.0;
#pragma unroll
    for (int q = 0; q < RM; ++q) {
        const int64_t i = r0 + tid + q * kGradThreads;
        const bool ok = i < p.n;
#pragma unroll
        for (int k = 0; k < D; ++k) xa[q][k] = ok ? p.Xs[i * D + k] : 0.0f;
        float g = 0.0f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            ua[q][c] = ok ? p.alpha[c] * p.U[i * C + c] : 0.0f;
            if (ok) g = fmaf(ua[q][c], p.V[i * C + c], g);
        }
        if (rank == 0) diag += (double)g;
    }
    float accf[NA - 1];
    double accd[NA - 1];
#pragma unroll
    for (int k = 0; k < NA - 1; ++k) { accf[k] = 0.0f; accd[k] = 0.0; }

    for (int64_t cb = c_lo; cb < c_hi; cb += kGradTN) {
        const int cnt = (int)min((int64_t)kGradTN, c_hi - cb);
        __syncthreads();
        for (int t = tid; t < cnt * D; t += kGradThreads) s_xb[t] = p.Xs[cb * D + t];
        for (int t = tid; t < cnt * C; t += kGradThreads) s_v[t] = p.V[cb * C + t];
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
#pragma unroll
            for (int q = 0; q < RM; ++q) {
                float df2[D];
                float t2 = 0.0f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const float df = xa[q][k] - s_xb[jj * D + k];
                    df2[k] = df * df;
                    t2 += df2[k];
                }
                float g = 0.0f;
#pragma unroll
                for (int c = 0; c < C; ++c) g = fmaf(ua[q][c], s_v[jj * C + c], g);
                float phi, psi;
                phi_psi_fp32<KERN>(t2, phi, psi);
                const float gp = g * psi;
#pragma unroll
                for (int k = 0; k < D; ++k) accf[k] = fmaf(gp, df2[k], accf[k]);
                accf[D] = fmaf(g, phi, accf[D]);
            }
        }
        // fold the chunk into FP64 so the n-term sums keep their precision
#pragma unroll
        for (int k = 0; k < NA - 1; ++k) { accd[k] += (double)accf[k]; accf[k] = 0.0f; }
    }
    // CTA sums in FP64, then the ticketed last CTA adds the partials in order
    for (int k = 0; k < NA; ++k) {
        const double v = k < NA - 1 ? accd[k] : diag;
        double t = cta_sum_d(v, red_d);
        if (tid == 0) s_tot[k] = t;
    }
    __syncthreads();
    const int64_t idx = (int64_t)blockIdx.x * S + rank;
    if (tid < NA) p.part[idx * NA + tid] = s_tot[tid];
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned total = (unsigned)(p.ntiles * S);
        s_last = (atomicAdd(p.ticket, 1u) == total - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int k = tid; k < NA; k += kGradThreads) {
            double acc = 0.0;
            for (int64_t t = 0; t < p.ntiles * S; ++t) acc += __ldcg(p.part + t * NA + k);
            p.out[k] = acc;
        }
        if (tid == 0) *p.ticket = 0u;
    }
}

template <int KERN, int D, int C>
cudaError_t launch_grad_inst(const GradParams& p, cudaStream_t st) {
    grad_kernel<KERN, D, C><<<dim3((unsigned)p.ntiles, (unsigned)p.S, 1), kGradThreads, 0, st>>>(p);
    return cudaGetLastError();
}

template <int KERN>
cudaError_t dispatch_grad(const GradParams& p, int D, int C, cudaStream_t st) {
#define AP_GRAD_C(DD)                                                    \
    switch (C) {                                                         \
        case 1: return launch_grad_inst<KERN, DD, 1>(p, st);             \
        case 4: return launch_grad_inst<KERN, DD, 4>(p, st);             \
        case 16: return launch_grad_inst<KERN, DD, 16>(p, st);           \
        case 32: return launch_grad_inst<KERN, DD, 32>(p, st);           \
        default: return cudaErrorInvalidValue;                           \
    }
    switch (D) {
        case 4: AP_GRAD_C(4)
        case 8: AP_GRAD_C(8)
        case 12: AP_GRAD_C(12)
        case 16: AP_GRAD_C(16)
        case 24: AP_GRAD_C(24)
        case 32: AP_GRAD_C(32)
        default: return cudaErrorInvalidValue;
    }
#undef AP_GRAD_C
}

}  // namespace ap
