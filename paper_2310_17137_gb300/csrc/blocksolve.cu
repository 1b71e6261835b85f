// Block solve of one AP step and small data-movement kernels.
//
// Delta = K_II^{-1} R_I = L^{-T} (L^{-1} R_I) and W_I += Delta (Alg. 1, the
// weight update Eq. text_update_of_w; Table 6: (b^2 + b) l flops).  I is read
// from device memory, where the previous step's epilogue left the
// Gauss-Southwell choice, so a whole epoch runs without a host round trip.
//
// Both triangular products are tiled by 64 x 64 tiles of the packed FP32
// inverse factor.  A thread-block cluster of S CTAs (S up to 16) shares one
// output tile; each CTA sums every S-th input tile and the S partial tiles are
// added through distributed shared memory in rank order (deterministic).  The
// next input tile is fetched into registers while the current one is used from
// shared memory, and each thread keeps one row and four columns per column
// quad in registers, so a 64 x 64 x C tile costs 64 (1 + C/16) shared loads per
// thread.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "ap_internal.cuh"

namespace ap {
namespace cg = cooperative_groups;
namespace {

constexpr int T = kTile;
constexpr int TP = kTile + 1;
constexpr int kSolveThreads = 256;
constexpr int kSolveMaxSplit = 16;  // non-portable cluster size, probed at launch

__device__ __forceinline__ int64_t packed_tile(int i, int k) { return (int64_t)i * (i + 1) / 2 + k; }

// Operand staging shared by both passes: one 64 x 64 tile of L^{-1} (16 float
// per thread) and one 64 x C tile of the right-hand side, padded to CP >= 4
// columns (at most two float4 per thread).
template <int C>
struct SolveTile {
    static constexpr int CP = C < 4 ? 4 : C;
    static constexpr int NQ = CP / 4;                                     // column quads
    static constexpr int NV = (T * CP / 4 + kSolveThreads - 1) / kSolveThreads;  // float4 of the RHS tile
    float4 x[4];
    float4 v[NV];

    __device__ __forceinline__ void load_x(const float* tile, int tid) {
        const float4* src = reinterpret_cast<const float4*>(tile);
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = __ldg(src + tid + j * kSolveThreads);
    }
    __device__ __forceinline__ void store_x(float* sx, int tid) const {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = tid + j * kSolveThreads;
            const int rr = (4 * t) / T, qq = (4 * t) % T;
            sx[rr * TP + qq + 0] = x[j].x;
            sx[rr * TP + qq + 1] = x[j].y;
            sx[rr * TP + qq + 2] = x[j].z;
            sx[rr * TP + qq + 3] = x[j].w;
        }
    }
    // RHS rows row0 .. row0 + 63 of an n x C matrix; rows >= nrows read as 0
    __device__ __forceinline__ void load_v(const float* M, int64_t row0, int64_t nrows, int tid) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int t = tid + j * kSolveThreads;  // float4 index within the 64 x CP tile
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (t < T * CP / 4) {
                const int rr = t / NQ, c4 = 4 * (t % NQ);
                if (row0 + rr < nrows) {
                    const float* src = M + (row0 + rr) * C + c4;
                    if constexpr (C >= 4) {
                        w = __ldg(reinterpret_cast<const float4*>(src));
                    } else {
                        w.x = __ldg(src);
                    }
                }
            }
            v[j] = w;
        }
    }
    __device__ __forceinline__ void store_v(float* sv, int tid) const {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int t = tid + j * kSolveThreads;
            if (t < T * CP / 4) reinterpret_cast<float4*>(sv)[t] = v[j];
        }
    }
};

// Fixed-order sum of the S partial tiles of a cluster (rank order); thread t
// of every rank finishes rows rank * 64 / S ... of the output tile.
template <int CP, typename F>
__device__ __forceinline__ void cluster_finish(float* spart, int S, int rank, int tid, F&& emit) {
    if (S > 1) cg::this_cluster().sync();
    else __syncthreads();
    const int rpr = T / S;
    for (int t = tid; t < rpr * CP; t += kSolveThreads) {
        const int rr = rank * rpr + t / CP, c = t % CP;
        float sum = 0.0f;
        if (S == 1) {
            sum = spart[rr * CP + c];
        } else {
            cg::cluster_group cl = cg::this_cluster();
            for (int src = 0; src < S; ++src) sum += cl.map_shared_rank(spart, src)[rr * CP + c];
        }
        emit(rr, c, sum);
    }
    if (S > 1) cg::this_cluster().sync();
}

// pass 1: Z_i = sum_{k <= i} X_ik R_I[k]  (X = L^{-1})
template <int C>
__global__ void __launch_bounds__(kSolveThreads) trmv_lower_kernel(const SolveParams p) {
    using Tl = SolveTile<C>;
    constexpr int CP = Tl::CP, NQ = Tl::NQ, QPT = (NQ + 3) / 4;  // column quads per thread
    __shared__ float sx[T * TP];
    __shared__ __align__(16) float sv[T * CP];
    __shared__ float spart[T * CP];
    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const int S = gridDim.y, rank = blockIdx.y;
    const int I = *p.sel;
    const int64_t lo = (int64_t)I * p.b;
    const int64_t bI = min(p.b, p.n - lo);
    const int64_t ntri = (int64_t)p.nt * (p.nt + 1) / 2;
    const float* Lb = p.Linv + (int64_t)I * ntri * T * T;
    const int r = tid % T, g = tid / T;  // output row, column-quad group
    float acc[QPT][4];
#pragma unroll
    for (int u = 0; u < QPT; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.0f;
    Tl op;
    if (rank <= i) {
        op.load_x(Lb + packed_tile(i, rank) * T * T, tid);
        op.load_v(p.R + lo * C, (int64_t)rank * T, bI, tid);
    }
    for (int k = rank; k <= i; k += S) {
        __syncthreads();
        op.store_x(sx, tid);
        op.store_v(sv, tid);
        __syncthreads();
        if (k + S <= i) {
            op.load_x(Lb + packed_tile(i, k + S) * T * T, tid);
            op.load_v(p.R + lo * C, (int64_t)(k + S) * T, bI, tid);
        }
#pragma unroll 8
        for (int q = 0; q < T; ++q) {
            const float xv = sx[r * TP + q];
#pragma unroll
            for (int u = 0; u < QPT; ++u) {
                const int quad = g + 4 * u;
                if (quad < NQ) {
                    const float4 w = reinterpret_cast<const float4*>(sv + q * CP)[quad];
                    acc[u][0] = fmaf(xv, w.x, acc[u][0]);
                    acc[u][1] = fmaf(xv, w.y, acc[u][1]);
                    acc[u][2] = fmaf(xv, w.z, acc[u][2]);
                    acc[u][3] = fmaf(xv, w.w, acc[u][3]);
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
        const int quad = g + 4 * u;
        if (quad < NQ)
#pragma unroll
            for (int j = 0; j < 4; ++j) spart[r * CP + 4 * quad + j] = acc[u][j];
    }
    cluster_finish<CP>(spart, S, rank, tid, [&](int rr, int c, float sum) {
        if (c < C) p.Z[((int64_t)i * T + rr) * C + c] = sum;
    });
}

// pass 2: Delta_k = sum_{i >= k} X_ik^T Z_i, then W_I += Delta.
template <int C>
__global__ void __launch_bounds__(kSolveThreads) trmv_upper_kernel(const SolveParams p) {
    using Tl = SolveTile<C>;
    constexpr int CP = Tl::CP, NQ = Tl::NQ, QPT = (NQ + 3) / 4;
    __shared__ float sx[T * TP];
    __shared__ __align__(16) float sv[T * CP];
    __shared__ float spart[T * CP];
    const int tid = threadIdx.x;
    const int k = blockIdx.x;
    const int S = gridDim.y, rank = blockIdx.y;
    const int I = *p.sel;
    const int64_t lo = (int64_t)I * p.b;
    const int64_t bI = min(p.b, p.n - lo);
    const int64_t ntri = (int64_t)p.nt * (p.nt + 1) / 2;
    const float* Lb = p.Linv + (int64_t)I * ntri * T * T;
    const int q = tid % T, g = tid / T;  // output row (column q of X), column-quad group
    const int64_t zrows = (int64_t)p.nt * T;
    float acc[QPT][4];
#pragma unroll
    for (int u = 0; u < QPT; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.0f;
    Tl op;
    if (k + rank < p.nt) {
        op.load_x(Lb + packed_tile(k + rank, k) * T * T, tid);
        op.load_v(p.Z, (int64_t)(k + rank) * T, zrows, tid);
    }
    for (int i = k + rank; i < p.nt; i += S) {
        __syncthreads();
        op.store_x(sx, tid);
        op.store_v(sv, tid);
        __syncthreads();
        if (i + S < p.nt) {
            op.load_x(Lb + packed_tile(i + S, k) * T * T, tid);
            op.load_v(p.Z, (int64_t)(i + S) * T, zrows, tid);
        }
#pragma unroll 8
        for (int rr = 0; rr < T; ++rr) {
            const float xv = sx[rr * TP + q];
#pragma unroll
            for (int u = 0; u < QPT; ++u) {
                const int quad = g + 4 * u;
                if (quad < NQ) {
                    const float4 w = reinterpret_cast<const float4*>(sv + rr * CP)[quad];
                    acc[u][0] = fmaf(xv, w.x, acc[u][0]);
                    acc[u][1] = fmaf(xv, w.y, acc[u][1]);
                    acc[u][2] = fmaf(xv, w.z, acc[u][2]);
                    acc[u][3] = fmaf(xv, w.w, acc[u][3]);
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
        const int quad = g + 4 * u;
        if (quad < NQ)
#pragma unroll
            for (int j = 0; j < 4; ++j) spart[q * CP + 4 * quad + j] = acc[u][j];
    }
    cluster_finish<CP>(spart, S, rank, tid, [&](int qq, int c, float sum) {
        if (c >= C) return;
        const int64_t li = (int64_t)k * T + qq;
        if (li < p.b) p.Delta[li * C + c] = li < bI ? sum : 0.0f;
        if (li < bI) p.W[(lo + li) * C + c] += sum;
    });
    if (k == 0 && rank == 0 && tid == 0 && p.trace) {
        const int64_t step = *p.step_ctr;
        if (step < p.trace_cap) p.trace[step] = I;
    }
}

// Largest cluster size S <= min(16, nt) (power of two) that the device can
// co-schedule for this kernel; 16 needs the non-portable opt-in.
template <typename K>
int solve_split(K kernel, int nt) {
    int S = 1;
    while (S * 2 <= kSolveMaxSplit && S * 2 <= nt) S *= 2;
    if (S > kMaxSplit) {
        bool ok = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
        if (ok) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)nt, (unsigned)S, 1);
            cfg.blockDim = dim3(kSolveThreads, 1, 1);
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 1;
            attr[0].val.clusterDim.y = (unsigned)S;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            ok = cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) == cudaSuccess && nclusters > 0;
        }
        cudaGetLastError();
        if (!ok) S = kMaxSplit;
    }
    return S;
}

// cluster size per (device, C, nt), probed once (contexts on several host
// threads share the table)
std::mutex g_split_mu;
std::map<std::tuple<int, int, int>, int> g_split;

template <int C>
int split_for(int nt) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    std::lock_guard<std::mutex> lk(g_split_mu);
    const auto key = std::make_tuple(dev, C, nt);
    auto it = g_split.find(key);
    if (it != g_split.end()) return it->second;
    const int S = std::min(solve_split(trmv_lower_kernel<C>, nt), solve_split(trmv_upper_kernel<C>, nt));
    g_split[key] = S;
    return S;
}

template <int C>
cudaError_t launch_solve_inst(const SolveParams& p, cudaStream_t st) {
    const int S = split_for<C>(p.nt);
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
