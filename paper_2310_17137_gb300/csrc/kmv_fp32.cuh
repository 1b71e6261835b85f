// FP32 SIMT form of the fused kernel-matrix product (the AP residual update,
// Eq. text_update_of_r, the residual recompute of the App. B lemma and the
// posterior mean of Sec. 2), with the block-norm / Gauss-Southwell epilogue of
// Eq. approximate_gauss_southwell fused in.
//
// Work decomposition
//   grid.x = row tiles of ROWS = 128 * RM rows; a tile never straddles an AP
//            block, so its squared norm belongs to exactly one block;
//   grid.y = S column splits, one thread-block cluster per row tile; the S
//            partial products are summed through distributed shared memory in
//            a fixed rank order (deterministic, no atomics on R).
// Each thread keeps RM rows of the scaled inputs and RM x C accumulators in
// registers; the block's columns (scaled inputs and the C right-hand sides of
// Delta) are staged through shared memory and read as warp broadcasts.  The
// n x b kernel block is never stored.
#pragma once

#include <cooperative_groups.h>

#include "ap_internal.cuh"

namespace ap {
namespace cg = cooperative_groups;

constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// phi as a function of t = |x_s - x_s'|^2 of the pre-scaled inputs.
template <int KERN>
__device__ __forceinline__ float phi_fp32(float t) {
    if constexpr (KERN == AP_RBF) {
        return ex2_approx(-t);
    } else if constexpr (KERN == AP_MATERN32) {
        float u = sqrt_approx(t);
        return (1.0f + u) * ex2_approx(-u * kLog2e);
    } else {
        float u = sqrt_approx(t);
        return fmaf(u, fmaf(u, 1.0f / 3.0f, 1.0f), 1.0f) * ex2_approx(-u * kLog2e);
    }
}

// SplitMix64 (Steele, Lea, Flood 2014; Vigna's reference constants) of
// (seed, counter): the counter-based stream behind AP_SEL_RANDOM.
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t idx) {
    uint64_t z = seed + (idx + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int random_block(uint64_t seed, int64_t step, int m) {
    uint64_t z = splitmix64_at(seed, (uint64_t)step);
    return (int)(((z >> 32) * (uint64_t)m) >> 32);
}

// Sum of one double over the CTA; the result is valid in thread 0.
__device__ __forceinline__ double cta_sum_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) r += red[i];
    return r;
}

// Executed by every thread of the CTA that finished last (ticket order):
// reduce the per-tile partials in a fixed order, pick the next block, publish
// the column norms, and leave the ticket at zero for the next launch.
template <int C>
__device__ void epi_finalize(const EpiParams& e, double* red_d, int* red_i) {
    const int tid = threadIdx.x, nth = blockDim.x;
    if (e.flags & kEpiBlockNorms) {
        double best = -1.0;
        int bi = 0x7fffffff;
        int bad = 0;
        const int64_t per = e.tiles_per_seg * e.S;
        for (int J = tid; J < e.m; J += nth) {
            double acc = 0.0;
            const double* src = e.part_norm + (int64_t)J * per;
            for (int64_t t = 0; t < per && AP_CHK((int64_t)J * per + t < e.ntiles * e.S); ++t) acc += __ldcg(src + t);
            e.norms_out[J] = acc;
            if (!isfinite(acc)) bad = 1;
            if (acc > best) { best = acc; bi = J; }
        }
        // argmax over the CTA, ties to the smallest block index
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_down_sync(0xffffffffu, best, o);
            int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        bad = __syncthreads_or(bad);
        const int w = tid >> 5, nw = nth >> 5;
        if ((tid & 31) == 0) { red_d[w] = best; red_i[w] = bi; }
        __syncthreads();
        if (tid == 0) {
            best = red_d[0];
            bi = red_i[0];
            for (int i = 1; i < nw; ++i)
                if (red_d[i] > best || (red_d[i] == best && red_i[i] < bi)) { best = red_d[i]; bi = red_i[i]; }
            int64_t step = *e.step_ctr + (e.advance ? 1 : 0);
            int next;
            if (e.select == AP_SEL_CYCLIC) next = (int)(step % e.m);
            else if (e.select == AP_SEL_RANDOM) next = random_block(e.seed, step, e.m);
            else next = (bi >= 0 && bi < e.m) ? bi : 0;
            *e.sel_out = next;
            *e.step_ctr = step;
            if (bad) *e.nan_flag = 1;
        }
        __syncthreads();
    }
    if (e.flags & kEpiColNorms) {
        const int64_t tot = e.ntiles * e.S;
        for (int c = tid; c < C; c += nth) {
            double acc = 0.0;
            for (int64_t t = 0; t < tot; ++t) acc += __ldcg(e.part_col + t * C + c);
            e.colnorm_out[c] = acc;
            if (!isfinite(acc)) *e.nan_flag = 1;
        }
    }
    if (tid == 0) *e.ticket = 0u;
}

// Phase 2 of every product: reduce the S rank partials of this CTA's share of
// rows (fixed rank order), add the base, store, and write the norm partials.
template <int C, int ROWS>
__device__ __forceinline__ void epi_store(const KmvParams& p, float* s_part, int S, int rank,
                                          int64_t r0, int64_t r1, int64_t part_idx, double* red_d,
                                          double* s_col) {
    const int tid = threadIdx.x;
    const int rpr = ROWS / S;  // rows reduced by this rank
    double sq = 0.0, colacc = 0.0;
    for (int t = tid; t < rpr * C; t += kKmvThreads) {
        const int lr = rank * rpr + t / C;
        const int c = t % C;  // == tid % C since kKmvThreads % C == 0
        const int64_t i = r0 + lr;
        float sum = 0.0f;
        if (S == 1) {
            sum = s_part[lr * C + c];
        } else {
            cg::cluster_group cluster = cg::this_cluster();
            for (int src = 0; src < S; ++src) {
                const float* peer = cluster.map_shared_rank(s_part, src);
                sum += peer[lr * C + c];
            }
        }
        if (i < r1 && AP_CHK(i < p.na)) {
            const float bv = p.base ? p.base[i * C + c] : p.base_const;
            const float o = fmaf(p.sgn, sum, bv);
            p.out[i * C + c] = o;
            const double od = (double)o;
            sq += od * od;
            colacc += od * od;
        }
    }
    const EpiParams& e = p.epi;
    if (e.flags & kEpiBlockNorms) {
        double tot = cta_sum_d(sq, red_d);
        if (tid == 0 && AP_CHK(part_idx < e.ntiles * e.S)) e.part_norm[part_idx] = tot;
    }
    if (e.flags & kEpiColNorms) {
        __syncthreads();
        s_col[tid] = colacc;
        __syncthreads();
        if (tid < C) {
            double acc = 0.0;
            for (int k = tid; k < kKmvThreads; k += C) acc += s_col[k];
            if (AP_CHK(part_idx < e.ntiles * e.S)) e.part_col[part_idx * C + tid] = acc;
        }
    }
}

template <int C>
__device__ __forceinline__ void epi_ticket(const EpiParams& e, double* red_d, int* red_i,
                                           int* s_last) {
    if (e.flags == 0) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned total = (unsigned)(e.ntiles * e.S);
        *s_last = (atomicAdd(e.ticket, 1u) == total - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (*s_last) {
        __threadfence();
        epi_finalize<C>(e, red_d, red_i);
    }
}

// With C a multiple of 4 the distance and the contraction run as packed FP32
// pairs (fma.rn.f32x2: one instruction for two lanes, each rounded as the scalar
// operation): the squared distance over pairs of coordinates (two partial sums,
// added at the end), the contraction over pairs of right-hand sides.  Shared
// memory holds the operands exactly as in the scalar form.
template <int C>
struct KmvPaired {
    static constexpr bool value = C % 4 == 0;
};

template <int D, int C, int RM>
constexpr size_t kmv_smem_floats() {
    return (size_t)kKmvTN * (D + C) + (size_t)kKmvThreads * RM * C;
}

template <int KERN, int D, int C, int RM>
__global__ void __launch_bounds__(kKmvThreads, 4) kmv_fp32_kernel(const KmvParams p) {
    constexpr int ROWS = kKmvThreads * RM;
    constexpr bool kPaired = KmvPaired<C>::value;
    extern __shared__ float4 kmv_smem4[];
    float* s_xb = reinterpret_cast<float*>(kmv_smem4);  // kKmvTN * D
    float* s_v = s_xb + kKmvTN * D;                     // kKmvTN * C
    float* s_part = s_v + kKmvTN * C;                   // ROWS * C
    __shared__ double red_d[32];
    __shared__ int red_i[32];
    __shared__ double s_col[kKmvThreads];
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int S = gridDim.y;
    const int rank = blockIdx.y;
    const EpiParams& e = p.epi;
    const int64_t tile = blockIdx.x;
    const int64_t segi = tile / e.tiles_per_seg;
    const int64_t seg_lo = segi * e.seg;
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

    float xa[RM][D];
#pragma unroll
    for (int q = 0; q < RM; ++q) {
        const int64_t i = r0 + tid + q * kKmvThreads;
#pragma unroll
        for (int k4 = 0; k4 < D / 4; ++k4) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < r1 && AP_CHK(i < p.na)) v = reinterpret_cast<const float4*>(p.Xa + i * D)[k4];
            xa[q][4 * k4 + 0] = v.x;
            xa[q][4 * k4 + 1] = v.y;
            xa[q][4 * k4 + 2] = v.z;
            xa[q][4 * k4 + 3] = v.w;
        }
    }
    float acc[RM][C];
#pragma unroll
    for (int q = 0; q < RM; ++q)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[q][c] = 0.0f;

    if constexpr (kPaired) {
        float2 xa2[RM][D / 2], acc2[RM][C / 2];
#pragma unroll
        for (int q = 0; q < RM; ++q) {
#pragma unroll
            for (int k = 0; k < D / 2; ++k) xa2[q][k] = make_float2(xa[q][2 * k], xa[q][2 * k + 1]);
#pragma unroll
            for (int c = 0; c < C / 2; ++c) acc2[q][c] = make_float2(0.0f, 0.0f);
        }
        const float2 m1 = make_float2(-1.0f, -1.0f);
        for (int64_t cb = c_lo; cb < c_hi; cb += kKmvTN) {
            const int cnt = (int)min((int64_t)kKmvTN, c_hi - cb);
            __syncthreads();
            if (AP_CHK(cb >= 0 && cb + cnt <= p.nb) && AP_CHK(cb - col0 >= 0 && cb - col0 + cnt <= ncols)) {
                const float4* gx = reinterpret_cast<const float4*>(p.Xb + cb * D);
                float4* sx = reinterpret_cast<float4*>(s_xb);
                for (int t = tid; t < cnt * D / 4; t += kKmvThreads) sx[t] = __ldg(gx + t);
                const float4* gv4 = reinterpret_cast<const float4*>(p.V + (cb - col0) * C);
                float4* sv4 = reinterpret_cast<float4*>(s_v);
                for (int t = tid; t < cnt * C / 4; t += kKmvThreads) sv4[t] = __ldg(gv4 + t);
            }
            __syncthreads();
#pragma unroll 2
            for (int jj = 0; jj < cnt; ++jj) {
                float2 xb2[D / 2];
#pragma unroll
                for (int k4 = 0; k4 < D / 4; ++k4) {
                    const float4 v = reinterpret_cast<const float4*>(s_xb + jj * D)[k4];
                    xb2[2 * k4] = make_float2(v.x, v.y);
                    xb2[2 * k4 + 1] = make_float2(v.z, v.w);
                }
                float kv[RM];
#pragma unroll
                for (int q = 0; q < RM; ++q) {
                    float2 tp = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int k = 0; k < D / 2; ++k) {
                        const float2 df = __ffma2_rn(xb2[k], m1, xa2[q][k]);  // xa - xb, exact negation
                        tp = __ffma2_rn(df, df, tp);
                    }
                    kv[q] = phi_fp32<KERN>(tp.x + tp.y);
                }
#pragma unroll
                for (int c4 = 0; c4 < C / 4; ++c4) {
                    const float4 v = reinterpret_cast<const float4*>(s_v + jj * C)[c4];
#pragma unroll
                    for (int q = 0; q < RM; ++q) {
                        const float2 kd = make_float2(kv[q], kv[q]);
                        acc2[q][2 * c4] = __ffma2_rn(kd, make_float2(v.x, v.y), acc2[q][2 * c4]);
                        acc2[q][2 * c4 + 1] = __ffma2_rn(kd, make_float2(v.z, v.w), acc2[q][2 * c4 + 1]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RM; ++q)
#pragma unroll
            for (int c = 0; c < C / 2; ++c) {
                acc[q][2 * c] = acc2[q][c].x;
                acc[q][2 * c + 1] = acc2[q][c].y;
            }
    } else
    for (int64_t cb = c_lo; cb < c_hi; cb += kKmvTN) {
        const int cnt = (int)min((int64_t)kKmvTN, c_hi - cb);
        __syncthreads();
        if (AP_CHK(cb >= 0 && cb + cnt <= p.nb) && AP_CHK(cb - col0 >= 0 && cb - col0 + cnt <= ncols)) {
            const float4* gx = reinterpret_cast<const float4*>(p.Xb + cb * D);
            float4* sx = reinterpret_cast<float4*>(s_xb);
            for (int t = tid; t < cnt * D / 4; t += kKmvThreads) sx[t] = __ldg(gx + t);
            const float* gv = p.V + (cb - col0) * C;
            if constexpr (C % 4 == 0) {
                const float4* gv4 = reinterpret_cast<const float4*>(gv);
                float4* sv4 = reinterpret_cast<float4*>(s_v);
                for (int t = tid; t < cnt * C / 4; t += kKmvThreads) sv4[t] = __ldg(gv4 + t);
            } else {
                for (int t = tid; t < cnt * C; t += kKmvThreads) s_v[t] = __ldg(gv + t);
            }
        }
        __syncthreads();
#pragma unroll 2
        for (int jj = 0; jj < cnt; ++jj) {
            float xb[D];
#pragma unroll
            for (int k4 = 0; k4 < D / 4; ++k4) {
                float4 v = reinterpret_cast<const float4*>(s_xb + jj * D)[k4];
                xb[4 * k4 + 0] = v.x;
                xb[4 * k4 + 1] = v.y;
                xb[4 * k4 + 2] = v.z;
                xb[4 * k4 + 3] = v.w;
            }
            float kv[RM];
#pragma unroll
            for (int q = 0; q < RM; ++q) {
                float t2 = 0.0f;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const float df = xa[q][k] - xb[k];
                    t2 = fmaf(df, df, t2);
                }
                kv[q] = phi_fp32<KERN>(t2);
            }
            if constexpr (C % 4 == 0) {
#pragma unroll
                for (int c4 = 0; c4 < C / 4; ++c4) {
                    const float4 v = reinterpret_cast<const float4*>(s_v + jj * C)[c4];
#pragma unroll
                    for (int q = 0; q < RM; ++q) {
                        acc[q][4 * c4 + 0] = fmaf(kv[q], v.x, acc[q][4 * c4 + 0]);
                        acc[q][4 * c4 + 1] = fmaf(kv[q], v.y, acc[q][4 * c4 + 1]);
                        acc[q][4 * c4 + 2] = fmaf(kv[q], v.z, acc[q][4 * c4 + 2]);
                        acc[q][4 * c4 + 3] = fmaf(kv[q], v.w, acc[q][4 * c4 + 3]);
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float v = s_v[jj * C + c];
#pragma unroll
                    for (int q = 0; q < RM; ++q) acc[q][c] = fmaf(kv[q], v, acc[q][c]);
                }
            }
        }
    }
    // scale by s, add sigma^2 V_i on the index diagonal, park in shared memory
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RM; ++q) {
        const int lr = tid + q * kKmvThreads;
        const int64_t i = r0 + lr;
        const bool diag = p.noise_diag && i >= c_lo && i < c_hi;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float v = p.s * acc[q][c];
            if (diag && AP_CHK(i - col0 >= 0 && i - col0 < ncols)) v = fmaf(p.noise, __ldg(p.V + (i - col0) * C + c), v);
            s_part[lr * C + c] = v;
        }
    }
    if (S > 1) cg::this_cluster().sync();
    else __syncthreads();
    epi_store<C, ROWS>(p, s_part, S, rank, r0, r1, tile * S + rank, red_d, s_col);
    if (S > 1) cg::this_cluster().sync();
    epi_ticket<C>(e, red_d, red_i, &s_last);
}

// Norms + selection of R alone (before the first step, after a refinement).
template <int C>
__global__ void __launch_bounds__(kKmvThreads) norms_select_kernel(const float* R, int64_t n,
                                                                   const EpiParams e,
                                                                   int64_t tile_rows) {
    __shared__ double red_d[32];
    __shared__ int red_i[32];
    __shared__ double s_col[kKmvThreads];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int64_t tile = blockIdx.x;
    const int64_t seg_lo = (tile / e.tiles_per_seg) * e.seg;
    const int64_t seg_hi = min(seg_lo + e.seg, n);
    const int64_t r0 = seg_lo + (tile % e.tiles_per_seg) * tile_rows;
    const int64_t r1 = min(r0 + tile_rows, seg_hi);
    double sq = 0.0, colacc = 0.0;
    for (int64_t t = tid; t < (r1 - r0) * C && AP_CHK(r1 <= n); t += kKmvThreads) {
        const double v = (double)R[r0 * C + t];
        sq += v * v;
        colacc += v * v;
    }
    if (e.flags & kEpiBlockNorms) {
        double tot = cta_sum_d(sq, red_d);
        if (tid == 0 && AP_CHK(tile < e.ntiles)) e.part_norm[tile] = tot;
    }
    if (e.flags & kEpiColNorms) {
        __syncthreads();
        s_col[tid] = colacc;
        __syncthreads();
        if (tid < C) {
            double acc = 0.0;
            for (int k = tid; k < kKmvThreads; k += C) acc += s_col[k];
            if (AP_CHK(tile < e.ntiles)) e.part_col[tile * C + tid] = acc;
        }
    }
    epi_ticket<C>(e, red_d, red_i, &s_last);
}

inline int rows_per_thread(int D, int C) {
    const int w = D + C;
    return w <= 20 ? 4 : (w <= 36 ? 2 : 1);
}

template <int KERN, int D, int C>
cudaError_t launch_kmv_inst(const KmvParams& p, cudaStream_t st) {
    constexpr int RM = (D + C <= 20) ? 4 : ((D + C <= 36) ? 2 : 1);
    const size_t smem = sizeof(float) * kmv_smem_floats<D, C, RM>();
    auto fn = kmv_fp32_kernel<KERN, D, C, RM>;
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

// (D, C) dispatch for one kernel family.
template <int KERN>
cudaError_t dispatch_kmv(const KmvParams& p, int D, int C, cudaStream_t st) {
#define AP_KMV_C(DD)                                                      \
    switch (C) {                                                          \
        case 1: return launch_kmv_inst<KERN, DD, 1>(p, st);               \
        case 4: return launch_kmv_inst<KERN, DD, 4>(p, st);               \
        case 16: return launch_kmv_inst<KERN, DD, 16>(p, st);             \
        case 32: return launch_kmv_inst<KERN, DD, 32>(p, st);             \
        default: return cudaErrorInvalidValue;                            \
    }
    switch (D) {
        case 4: AP_KMV_C(4)
        case 8: AP_KMV_C(8)
        case 12: AP_KMV_C(12)
        case 16: AP_KMV_C(16)
        case 24: AP_KMV_C(24)
        case 32: AP_KMV_C(32)
        default: return cudaErrorInvalidValue;
    }
#undef AP_KMV_C
}

}  // namespace ap
