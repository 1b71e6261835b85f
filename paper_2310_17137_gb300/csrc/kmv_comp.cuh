// Compensated FP32 form of the kernel-matrix product, used to recompute the
// residual R = B - K_hat W for refinement when the requested tolerance is
// below what plain FP32 kernel entries can certify.
//
// Every quantity is a double-float (FP32 pair): the scaled inputs carry their
// rounding remainders (x_s = hi + lo), the squared distance is summed exactly
// enough (TwoSum of the coordinate differences, TwoProd of the squares), phi
// is evaluated with the double-float exp2 / sqrt of dfloat.cuh, and the
// products with V are accumulated with TwoProd + double-float additions.  The
// entries then carry ~1e-11 relative error instead of ~3e-7.  Same grid, same
// fixed-order cluster reduction and the same epilogue as the plain form.
#pragma once

#include "dfloat.cuh"
#include "kmv_fp32.cuh"

namespace ap {

template <int KERN>
__device__ __forceinline__ df::F2 phi_df(df::F2 t) {
    if constexpr (KERN == AP_RBF) {
        return df::exp2_neg(t);
    } else {
        const df::F2 u = df::sqrt_df(t);
        const df::F2 e = df::exp2_neg(df::mul(u, df::F2{df::kLog2eH, df::kLog2eL}));
        df::F2 poly = df::add_f(u, 1.0f);
        if constexpr (KERN == AP_MATERN52) {
            const df::F2 u2 = df::mul(u, u);
            poly = df::add(poly, df::mul(u2, df::F2{df::kThirdH, df::kThirdL}));
        }
        return df::mul(poly, e);
    }
}

template <int KERN, int D, int C>
__global__ void __launch_bounds__(kKmvThreads) kmv_comp_kernel(const KmvParams p) {
    constexpr int ROWS = kCompRows;
    extern __shared__ float4 kc_smem4[];
    float* s_xh = reinterpret_cast<float*>(kc_smem4);  // kKmvTN * D
    float* s_xl = s_xh + kKmvTN * D;                  // kKmvTN * D
    float* s_v = s_xl + kKmvTN * D;                   // kKmvTN * C
    float* s_ph = s_v + kKmvTN * C;                   // ROWS * C
    float* s_pl = s_ph + ROWS * C;                    // ROWS * C
    __shared__ double red_d[32];
    __shared__ int red_i[32];
    __shared__ double s_col[kKmvThreads];
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int S = gridDim.y;
    const int rank = blockIdx.y;
    const EpiParams& e = p.epi;
    const int64_t tile = blockIdx.x;
    const int64_t seg_lo = (tile / e.tiles_per_seg) * e.seg;
    const int64_t seg_hi = min(seg_lo + e.seg, p.na);
    const int64_t r0 = seg_lo + (tile % e.tiles_per_seg) * ROWS;
    const int64_t r1 = min(r0 + (int64_t)ROWS, seg_hi);
    int64_t col0 = p.col0, ncols = p.ncols;
    if (p.sel) {
        col0 = (int64_t)(*p.sel) * p.blk;
        ncols = min(p.blk, p.nb - col0);
    }
    const int64_t cs = ((ncols + S - 1) / S + kKmvTN - 1) / kKmvTN * kKmvTN;
    const int64_t c_lo = col0 + rank * cs;
    const int64_t c_hi = min(col0 + ncols, c_lo + cs);

    const int64_t i = r0 + tid;
    const bool live = i < r1 && AP_CHK(i < p.na);
    float xh[D], xl[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        xh[k] = live ? p.Xa[i * D + k] : 0.0f;
        xl[k] = live ? p.Xa_lo[i * D + k] : 0.0f;
    }
    df::F2 acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = {0.0f, 0.0f};

    for (int64_t cb = c_lo; cb < c_hi; cb += kKmvTN) {
        const int cnt = (int)min((int64_t)kKmvTN, c_hi - cb);
        __syncthreads();
        if (AP_CHK(cb >= 0 && cb + cnt <= p.nb) && AP_CHK(cb - col0 >= 0 && cb - col0 + cnt <= ncols)) {
            for (int t = tid; t < cnt * D; t += kKmvThreads) {
                s_xh[t] = p.Xb[cb * D + t];
                s_xl[t] = p.Xb_lo[cb * D + t];
            }
            for (int t = tid; t < cnt * C; t += kKmvThreads) s_v[t] = p.V[(cb - col0) * C + t];
        }
        __syncthreads();
        for (int jj = 0; jj < cnt; ++jj) {
            df::F2 t2 = {0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < D; ++k) {
                df::F2 dh = df::two_sum(xh[k], -s_xh[jj * D + k]);
                dh = df::fast_two_sum(dh.h, dh.l + (xl[k] - s_xl[jj * D + k]));
                t2 = df::add(t2, df::mul(dh, dh));
            }
            const df::F2 kv = phi_df<KERN>(t2);
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = df::add(acc[c], df::mul_f(kv, s_v[jj * C + c]));
        }
    }
    __syncthreads();
    const bool diag = live && p.noise_diag && i >= c_lo && i < c_hi;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        df::F2 v = df::mul_f(acc[c], p.s);
        if (diag && AP_CHK(i - col0 >= 0 && i - col0 < ncols)) v = df::add(v, df::two_prod(p.noise, p.V[(i - col0) * C + c]));
        s_ph[tid * C + c] = v.h;
        s_pl[tid * C + c] = v.l;
    }
    if (S > 1) cg::this_cluster().sync();
    else __syncthreads();
    // fixed-order reduction of the S double-float partials, then the common epilogue
    const int rpr = ROWS / S;
    double sq = 0.0, colacc = 0.0;
    for (int t = tid; t < rpr * C; t += kKmvThreads) {
        const int lr = rank * rpr + t / C;
        const int c = t % C;
        const int64_t ii = r0 + lr;
        df::F2 sum = {s_ph[lr * C + c], s_pl[lr * C + c]};
        if (S > 1) {
            cg::cluster_group cluster = cg::this_cluster();
            sum = {0.0f, 0.0f};
            for (int src = 0; src < S; ++src)
                sum = df::add(sum, df::F2{cluster.map_shared_rank(s_ph, src)[lr * C + c],
                                          cluster.map_shared_rank(s_pl, src)[lr * C + c]});
        }
        if (ii < r1 && AP_CHK(ii < p.na)) {
            const float bv = p.base ? p.base[ii * C + c] : p.base_const;
            const df::F2 o2 = df::add_f(df::F2{p.sgn * sum.h, p.sgn * sum.l}, bv);
            const float o = o2.h + o2.l;
            p.out[ii * C + c] = o;
            const double od = (double)o;
            sq += od * od;
            colacc += od * od;
        }
    }
    if (e.flags & kEpiBlockNorms) {
        double tot = cta_sum_d(sq, red_d);
        if (tid == 0 && AP_CHK(tile * S + rank < e.ntiles * e.S)) e.part_norm[tile * S + rank] = tot;
    }
    if (e.flags & kEpiColNorms) {
        __syncthreads();
        s_col[tid] = colacc;
        __syncthreads();
        if (tid < C) {
            double a = 0.0;
            for (int k = tid; k < kKmvThreads; k += C) a += s_col[k];
            if (AP_CHK(tile * S + rank < e.ntiles * e.S)) e.part_col[(tile * S + rank) * C + tid] = a;
        }
    }
    if (S > 1) cg::this_cluster().sync();
    epi_ticket<C>(e, red_d, red_i, &s_last);
}

template <int KERN, int D, int C>
cudaError_t launch_kmv_comp_inst(const KmvParams& p, cudaStream_t st) {
    const size_t smem = sizeof(float) * ((size_t)kKmvTN * (2 * D + C) + (size_t)2 * kCompRows * C);
    auto fn = kmv_comp_kernel<KERN, D, C>;
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int S = p.epi.S;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.epi.ntiles, (unsigned)S, 1);
    cfg.blockDim = dim3(kKmvThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (S > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1;
        attr[0].val.clusterDim.y = (unsigned)S;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, fn, p);
}

template <int KERN>
cudaError_t dispatch_kmv_comp(const KmvParams& p, int D, int C, cudaStream_t st) {
#define AP_KMVC_C(DD)                                                       \
    switch (C) {                                                            \
        case 1: return launch_kmv_comp_inst<KERN, DD, 1>(p, st);            \
        case 4: return launch_kmv_comp_inst<KERN, DD, 4>(p, st);            \
        case 16: return launch_kmv_comp_inst<KERN, DD, 16>(p, st);          \
        case 32: return launch_kmv_comp_inst<KERN, DD, 32>(p, st);          \
        default: return cudaErrorInvalidValue;                              \
    }
    switch (D) {
        case 4: AP_KMVC_C(4)
        case 8: AP_KMVC_C(8)
        case 12: AP_KMVC_C(12)
        case 16: AP_KMVC_C(16)
        case 24: AP_KMVC_C(24)
        case 32: AP_KMVC_C(32)
        default: return cudaErrorInvalidValue;
    }
#undef AP_KMVC_C
}

}  // namespace ap
