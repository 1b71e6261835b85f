// Block solve of one AP step and small data-movement kernels.
//
// Delta = K_II^{-1} R_I = L^{-T} (L^{-1} R_I) and W_I += Delta (Alg. 1, the
// weight update Eq. text_update_of_w; Table 6: (b^2 + b) l flops).  I is read
// from device memory, where the previous step's epilogue left the
// Gauss-Southwell choice, so a whole epoch runs without a host round trip.
//
// Both triangular products are tiled by 64 x 64 tiles of the packed FP32
// inverse factor.  A thread-block cluster of S CTAs shares one output tile;
// each CTA sums every S-th input tile and the S partial tiles are added
// through distributed shared memory in rank order (deterministic).
#include <cooperative_groups.h>

#include "ap_internal.cuh"

namespace ap {
namespace cg = cooperative_groups;
namespace {

constexpr int T = kTile;
constexpr int TP = kTile + 1;
constexpr int kSolveThreads = 256;

__device__ __forceinline__ int64_t packed_tile(int i, int k) { return (int64_t)i * (i + 1) / 2 + k; }

// pass 1: Z_i = sum_{k <= i} X_ik R_I[k]  (X = L^{-1})
template <int C>
__global__ void __launch_bounds__(kSolveThreads) trmv_lower_kernel(const SolveParams p) {
    __shared__ float sx[T * TP];
    __shared__ float sr[T * C];
    __shared__ float spart[T * C];
    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const int S = gridDim.y, rank = blockIdx.y;
    const int I = *p.sel;
    const int64_t lo = (int64_t)I * p.b;
    const int64_t bI = min(p.b, p.n - lo);
    const int64_t ntri = (int64_t)p.nt * (p.nt + 1) / 2;
    const float* Lb = p.Linv + (int64_t)I * ntri * T * T;
    const int r = tid % T, g = tid / T;  // output row, column group
    constexpr int NC = (C + 3) / 4;
    float acc[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) acc[u] = 0.0f;
    for (int k = rank; k <= i; k += S) {
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(Lb + packed_tile(i, k) * T * T);
        for (int t = tid; t < T * T / 4; t += kSolveThreads) {
            const float4 v = __ldg(src + t);
            const int rr = (4 * t) / T, qq = (4 * t) % T;
            sx[rr * TP + qq + 0] = v.x;
            sx[rr * TP + qq + 1] = v.y;
            sx[rr * TP + qq + 2] = v.z;
            sx[rr * TP + qq + 3] = v.w;
        }
        for (int t = tid; t < T * C; t += kSolveThreads) {
            const int64_t li = (int64_t)k * T + t / C;
            sr[t] = li < bI ? p.R[(lo + li) * C + t % C] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NC; ++u) {
            const int c = g + 4 * u;
            if (c < C) {
                float a = acc[u];
                for (int q = 0; q < T; ++q) a = fmaf(sx[r * TP + q], sr[q * C + c], a);
                acc[u] = a;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NC; ++u) {
        const int c = g + 4 * u;
        if (c < C) spart[r * C + c] = acc[u];
    }
    if (S > 1) cg::this_cluster().sync();
    else __syncthreads();
    const int rpr = T / S;
    for (int t = tid; t < rpr * C; t += kSolveThreads) {
        const int rr = rank * rpr + t / C, c = t % C;
        float sum = 0.0f;
        if (S == 1) {
            sum = spart[rr * C + c];
        } else {
            cg::cluster_group cl = cg::this_cluster();
            for (int src = 0; src < S; ++src) sum += cl.map_shared_rank(spart, src)[rr * C + c];
        }
        p.Z[((int64_t)i * T + rr) * C + c] = sum;
    }
    if (S > 1) cg::this_cluster().sync();
}

// pass 2: Delta_k = sum_{i >= k} X_ik^T Z_i, then W_I += Delta.
template <int C>
__global__ void __launch_bounds__(kSolveThreads) trmv_upper_kernel(const SolveParams p) {
    __shared__ float sx[T * TP];
    __shared__ float sz[T * C];
    __shared__ float spart[T * C];
    const int tid = threadIdx.x;
    const int k = blockIdx.x;
    const int S = gridDim.y, rank = blockIdx.y;
    const int I = *p.sel;
    const int64_t lo = (int64_t)I * p.b;
    const int64_t bI = min(p.b, p.n - lo);
    const int64_t ntri = (int64_t)p.nt * (p.nt + 1) / 2;
    const float* Lb = p.Linv + (int64_t)I * ntri * T * T;
    const int q = tid % T, g = tid / T;
    constexpr int NC = (C + 3) / 4;
    float acc[NC];
#pragma unroll
    for (int u = 0; u < NC; ++u) acc[u] = 0.0f;
    for (int i = k + rank; i < p.nt; i += S) {
        __syncthreads();
        const float4* src = reinterpret_cast<const float4*>(Lb + packed_tile(i, k) * T * T);
        for (int t = tid; t < T * T / 4; t += kSolveThreads) {
            const float4 v = __ldg(src + t);
            const int rr = (4 * t) / T, qq = (4 * t) % T;
            sx[rr * TP + qq + 0] = v.x;
            sx[rr * TP + qq + 1] = v.y;
            sx[rr * TP + qq + 2] = v.z;
            sx[rr * TP + qq + 3] = v.w;
        }
        for (int t = tid; t < T * C; t += kSolveThreads) sz[t] = p.Z[(int64_t)i * T * C + t];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NC; ++u) {
            const int c = g + 4 * u;
            if (c < C) {
                float a = acc[u];
                for (int rr = 0; rr < T; ++rr) a = fmaf(sx[rr * TP + q], sz[rr * C + c], a);
                acc[u] = a;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NC; ++u) {
        const int c = g + 4 * u;
        if (c < C) spart[q * C + c] = acc[u];
    }
    if (S > 1) cg::this_cluster().sync();
    else __syncthreads();
    const int rpr = T / S;
    for (int t = tid; t < rpr * C; t += kSolveThreads) {
        const int qq = rank * rpr + t / C, c = t % C;
        float sum = 0.0f;
        if (S == 1) {
            sum = spart[qq * C + c];
        } else {
            cg::cluster_group cl = cg::this_cluster();
            for (int src = 0; src < S; ++src) sum += cl.map_shared_rank(spart, src)[qq * C + c];
        }
        const int64_t li = (int64_t)k * T + qq;
        if (li < p.b) p.Delta[li * C + c] = li < bI ? sum : 0.0f;
        if (li < bI) p.W[(lo + li) * C + c] += sum;
    }
    if (k == 0 && rank == 0 && tid == 0 && p.trace) {
        const int64_t step = *p.step_ctr;
        if (step < p.trace_cap) p.trace[step] = I;
    }
    if (S > 1) cg::this_cluster().sync();
}

template <int C>
cudaError_t launch_solve_inst(const SolveParams& p, cudaStream_t st) {
    int S = 1;
    while (S * 2 <= kMaxSplit && S * 2 <= p.nt) S *= 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.nt, (unsigned)S, 1);
    cfg.blockDim = dim3(kSolveThreads, 1, 1);
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
    cudaError_t err = cudaLaunchKernelEx(&cfg, trmv_lower_kernel<C>, p);
    if (err != cudaSuccess) return err;
    return cudaLaunchKernelEx(&cfg, trmv_upper_kernel<C>, p);
}

}  // namespace

cudaError_t launch_block_solve(const SolveParams& p, cudaStream_t st, int64_t* launches) {
    if (launches) *launches += 2;
    switch (p.C) {
        case 1: return launch_solve_inst<1>(p, st);
        case 4: return launch_solve_inst<4>(p, st);
        case 16: return launch_solve_inst<16>(p, st);
        case 32: return launch_solve_inst<32>(p, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ap
