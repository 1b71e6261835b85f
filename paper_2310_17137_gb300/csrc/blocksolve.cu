// Block solve of one AP step.
//
// Delta = K_II^{-1} R_I = L^{-T} (L^{-1} R_I) and W_I += Delta (Alg. 1, the
// weight update Eq. text_update_of_w; Table 6: (b^2 + b) l flops).  I is read
// from device memory, where the previous step's epilogue left the
// Gauss-Southwell choice, so a whole epoch runs without a host round trip.
//
// Both triangular products run over the 64 x 64 tiles of the packed FP32
// inverse factor (nt (nt + 1) / 2 tiles, read once per pass).  The tiles are
// split evenly over the CTAs (tpc consecutive tiles each: row-major order for
// Z = L^{-1} R_I, column-major for Delta = L^{-T} Z), so that every CTA reads
// the same number of bytes whatever the row lengths.  A CTA whose range covers
// part of an output row (of tiles) writes its partial sums to a slot of that
// row; the CTA that arrives last at the row's ticket adds the slots in slot
// order (deterministic) and writes the row.  Within a CTA the next tile is
// fetched into registers while the current one is used from shared memory, and
// each thread keeps one row and four columns per column quad in registers.
#include <algorithm>

#include "ap_internal.cuh"

namespace ap {
namespace {

constexpr int T = kTile;
constexpr int TP = kTile + 1;
constexpr int kSolveThreads = 256;

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

// Work split shared by host and device: tiles per CTA and partial slots per
// output row.
__host__ __device__ inline int64_t solve_ntri(int nt) { return (int64_t)nt * (nt + 1) / 2; }

// first tile of column k in column-major order of the lower triangle
__host__ __device__ inline int64_t col_start(int nt, int k) { return (int64_t)k * nt - (int64_t)k * (k - 1) / 2; }

// Partial sums of one output row (of tiles) from this CTA: write the slot, take
// a ticket, and if this CTA is the last of the row's `nslots` contributors, add
// the slots in order and hand each sum to emit(row-in-tile, column, value).
template <int CP, int QPT, typename F>
__device__ __forceinline__ void flush_row(const SolveParams& p, int row, int slot, int nslots,
                                          const float (&acc)[QPT][4], int r, int g, int* s_last, F&& emit) {
    constexpr int NQ = CP / 4;
    float* dst = p.spart + ((int64_t)row * p.maxj + slot) * T * CP;
    const bool slot_ok = AP_CHK(slot >= 0 && slot < p.maxj && nslots <= p.maxj && row < p.nt);
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
        const int quad = g + 4 * u;
        if (quad < NQ && slot_ok)
            *reinterpret_cast<float4*>(dst + r * CP + 4 * quad) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_last = (atomicAdd(p.sticket + row, 1u) == (unsigned)(nslots - 1)) ? 1 : 0;
    __syncthreads();
    if (*s_last) {
        __threadfence();
        const float* src = p.spart + (int64_t)row * p.maxj * T * CP;
        constexpr int EPT = T * CP / kSolveThreads;  // elements per thread
        float sum[EPT];
#pragma unroll
        for (int x = 0; x < EPT; ++x) sum[x] = 0.0f;
        // slots in order, eight at a time with all their loads in flight
        for (int j0 = 0; j0 < nslots; j0 += 8) {
            float v[8][EPT];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
#pragma unroll
                for (int x = 0; x < EPT; ++x)
                    v[jj][x] = j0 + jj < nslots
                                   ? __ldcg(src + (int64_t)(j0 + jj) * T * CP + threadIdx.x + x * kSolveThreads)
                                   : 0.0f;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
#pragma unroll
                for (int x = 0; x < EPT; ++x) sum[x] += v[jj][x];
        }
#pragma unroll
        for (int x = 0; x < EPT; ++x) {
            const int e = threadIdx.x + x * kSolveThreads;
            emit(e / CP, e % CP, sum[x]);
        }
        if (threadIdx.x == 0) p.sticket[row] = 0u;
    }
    __syncthreads();
}

// pass 1: Z_i = sum_{k <= i} X_ik R_I[k]  (X = L^{-1}), tiles in row-major order
template <int C>
__global__ void __launch_bounds__(kSolveThreads) solve_lower_kernel(const SolveParams p) {
    using Tl = SolveTile<C>;
    constexpr int CP = Tl::CP, NQ = Tl::NQ, QPT = (NQ + 3) / 4;
    __shared__ float sx[T * TP];
    __shared__ __align__(16) float sv[T * CP];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int I = *p.sel;
    const int64_t lo = (int64_t)I * p.b;
    if (!AP_CHK(I >= 0 && lo < p.n)) return;
    const int64_t bI = min(p.b, p.n - lo);
    const int64_t ntri = solve_ntri(p.nt);
    const float* Lb = p.Linv + (int64_t)I * ntri * T * T;
    const int64_t t0 = (int64_t)blockIdx.x * p.tpc, t1 = min(t0 + p.tpc, ntri);
    const int r = tid % T, g = tid / T;
    int i = 0;
    while (packed_tile(i + 1, 0) <= t0) ++i;
    int k = (int)(t0 - packed_tile(i, 0));
    float acc[QPT][4];
#pragma unroll
    for (int u = 0; u < QPT; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.0f;
    Tl op;
    op.load_x(Lb + t0 * T * T, tid);
    op.load_v(p.R + lo * C, (int64_t)k * T, bI, tid);
    for (int64_t t = t0; t < t1; ++t) {
        __syncthreads();
        op.store_x(sx, tid);
        op.store_v(sv, tid);
        __syncthreads();
        const int ni = k == i ? i + 1 : i, nk = k == i ? 0 : k + 1;
        if (t + 1 < t1) {
            op.load_x(Lb + (t + 1) * T * T, tid);
            op.load_v(p.R + lo * C, (int64_t)nk * T, bI, tid);
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
        if (k == i || t + 1 == t1) {
            const int first = (int)(packed_tile(i, 0) / p.tpc), last = (int)((packed_tile(i, 0) + i) / p.tpc);
            flush_row<CP, QPT>(p, i, (int)blockIdx.x - first, last - first + 1, acc, r, g, &s_last,
                               [&](int rr, int c, float sum) {
                                   if (c < C) p.Z[((int64_t)i * T + rr) * C + c] = sum;
                               });
#pragma unroll
            for (int u = 0; u < QPT; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.0f;
        }
        i = ni;
        k = nk;
    }
}

// pass 2: Delta_k = sum_{i >= k} X_ik^T Z_i, then W_I += Delta; tiles in
// column-major order
template <int C>
__global__ void __launch_bounds__(kSolveThreads) solve_upper_kernel(const SolveParams p) {
    using Tl = SolveTile<C>;
    constexpr int CP = Tl::CP, NQ = Tl::NQ, QPT = (NQ + 3) / 4;
    __shared__ float sx[T * TP];
    __shared__ __align__(16) float sv[T * CP];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int I = *p.sel;
    const int nt = p.nt;
    const int64_t lo = (int64_t)I * p.b;
    if (!AP_CHK(I >= 0 && lo < p.n)) return;
    const int64_t bI = min(p.b, p.n - lo);
    const int64_t ntri = solve_ntri(nt);
    const float* Lb = p.Linv + (int64_t)I * ntri * T * T;
    const int64_t zrows = (int64_t)nt * T;
    const int64_t u0 = (int64_t)blockIdx.x * p.tpc, u1 = min(u0 + p.tpc, ntri);
    const int q = tid % T, g = tid / T;
    int k = 0;
    while (col_start(nt, k + 1) <= u0) ++k;
    int i = k + (int)(u0 - col_start(nt, k));
    float acc[QPT][4];
#pragma unroll
    for (int u = 0; u < QPT; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.0f;
    Tl op;
    op.load_x(Lb + packed_tile(i, k) * T * T, tid);
    op.load_v(p.Z, (int64_t)i * T, zrows, tid);
    for (int64_t u = u0; u < u1; ++u) {
        __syncthreads();
        op.store_x(sx, tid);
        op.store_v(sv, tid);
        __syncthreads();
        const int nk = i == nt - 1 ? k + 1 : k, ni = i == nt - 1 ? k + 1 : i + 1;
        if (u + 1 < u1) {
            op.load_x(Lb + packed_tile(ni, nk) * T * T, tid);
            op.load_v(p.Z, (int64_t)ni * T, zrows, tid);
        }
#pragma unroll 8
        for (int rr = 0; rr < T; ++rr) {
            const float xv = sx[rr * TP + q];
#pragma unroll
            for (int uu = 0; uu < QPT; ++uu) {
                const int quad = g + 4 * uu;
                if (quad < NQ) {
                    const float4 w = reinterpret_cast<const float4*>(sv + rr * CP)[quad];
                    acc[uu][0] = fmaf(xv, w.x, acc[uu][0]);
                    acc[uu][1] = fmaf(xv, w.y, acc[uu][1]);
                    acc[uu][2] = fmaf(xv, w.z, acc[uu][2]);
                    acc[uu][3] = fmaf(xv, w.w, acc[uu][3]);
                }
            }
        }
        if (i == nt - 1 || u + 1 == u1) {
            const int first = (int)(col_start(nt, k) / p.tpc), last = (int)((col_start(nt, k) + nt - 1 - k) / p.tpc);
            const int kk = k;
            flush_row<CP, QPT>(p, k, (int)blockIdx.x - first, last - first + 1, acc, q, g, &s_last,
                               [&](int qq, int c, float sum) {
                                   if (c >= C) return;
                                   const int64_t li = (int64_t)kk * T + qq;
                                   if (li < p.b) p.Delta[li * C + c] = li < bI ? sum : 0.0f;
                                   if (li < bI && AP_CHK(lo + li < p.n)) p.W[(lo + li) * C + c] += sum;
                               });
#pragma unroll
            for (int uu = 0; uu < QPT; ++uu) acc[uu][0] = acc[uu][1] = acc[uu][2] = acc[uu][3] = 0.0f;
        }
        i = ni;
        k = nk;
    }
    if (blockIdx.x == 0 && tid == 0 && p.trace) {
        const int64_t step = *p.step_ctr;
        if (step < p.trace_cap) p.trace[step] = I;
    }
}

template <int C>
cudaError_t launch_solve_inst(const SolveParams& p, cudaStream_t st) {
    const unsigned grid = (unsigned)((solve_ntri(p.nt) + p.tpc - 1) / p.tpc);
    solve_lower_kernel<C><<<grid, kSolveThreads, 0, st>>>(p);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    solve_upper_kernel<C><<<grid, kSolveThreads, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

void block_solve_layout(int nt, int num_sms, int* tpc, int* maxj) {
    const int64_t target = 8LL * std::max(1, num_sms);
    *tpc = (int)std::max<int64_t>(1, (solve_ntri(nt) + target - 1) / target);
    *maxj = (nt + *tpc - 1) / *tpc + 1;
}

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
