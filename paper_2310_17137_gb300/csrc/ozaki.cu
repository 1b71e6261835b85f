// Trailing update of the tiled FP64 Cholesky (Sec. 3, "Cached Cholesky
// Factors"; the SYRK/GEMM step carries b^3/3 of the factorisation's flops) and
// its panel solve (TRSM as the product A_ik L_kk^{-T}) on the tensor cores,
// with FP64 results.
//
// A_ij -= A_ik A_jk^T for the trailing tiles k < j <= i is an FP64 dot product
// of length 64 per entry.  GB300 runs FP64 at about 2 FMA per clock per SM, so
// the products are formed as exact integer arithmetic on the BF16 tensor cores
// instead (the splitting scheme of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication", Numer. Algorithms 2012):
//   1. every row r of the 64-wide panel is scaled by a power of two 2^-e_r so
//      that its entries lie in (-1/2, 1/2), and each scaled entry x is written
//      as x = sum_{p=1..8} s_p 2^{-7p} + rest, |rest| < 2^-57, with integer
//      slices |s_p| <= 64 (exact in BF16);
//   2. for every level L = p + q = 2..9 the tensor cores accumulate
//      acc_L = sum_{p+q=L} sum_kk s_p(r, kk) s_q(c, kk) in FP32.  Every partial
//      sum is an integer below 2^22, so the accumulation is exact;
//   3. the levels are combined exactly in 64-bit integers,
//      H = sum_{L<=5} acc_L 2^{7(5-L)}, Lo = sum_{L>=6} acc_L 2^{7(9-L)}, and
//      A_rc -= 2^{e_r+e_c-35} (H + 2^-28 Lo) with two FP64 roundings.
// The terms left out (levels above 9 and the slice remainders) are below about
// 2^-50 K max_kk|a_r,kk| max_kk|a_c,kk| per entry, the size of FP64 rounding
// when the entries of a panel row have similar magnitudes; the matrix itself
// stays FP64.  On kernel blocks the factor's backward error ||L L^T - K|| / ||K||
// matches the all-FP64 factorisation (6e-16 vs 5e-16 on a Matern-5/2 block
// with condition number 1.6e4, in a NumPy model of these exact steps).
//
// Work item: a 128 x 64 output super-tile (two row tiles i0, i0 + 1 against
// one column tile j) of one block: bulk copies of the 8 slice planes of both
// operands (192 KB of shared memory), 144 MMAs (36 slice products x 4 K-steps
// of 16) into eight 64-column FP32 accumulators (all 512 tensor-memory
// columns), then an epilogue of one row per thread.  One persistent CTA per SM
// walks the work items; the next item's slices are copied in while the
// epilogue of the current one runs.  Every wait is bounded.
#include <cuda_bf16.h>

#include <algorithm>

#include "ap_internal.cuh"
#include "tcgen05.cuh"

namespace ap {
namespace {

using namespace tc;

constexpr int T = kTile;
constexpr int kSlices = 8;
constexpr int kSlabRows = 2 * T;                            // rows of a super-tile
constexpr uint32_t kPlaneA = kSlabRows * T * 2;             // 16 KB of BF16
constexpr uint32_t kPlaneB = T * T * 2;                     // 8 KB
constexpr uint32_t kOzSmem = kSlices * (kPlaneA + kPlaneB); // 192 KB
constexpr int kOzThreads = 256;  // 8 warps: two per tensor-memory lane quarter
constexpr uint32_t kRowBytes = T * 2;                       // one slice row (64 BF16)
constexpr int kBadExp = -(1 << 30);  // row exponent marking a non-finite panel row

// byte offset of (row, kk) in a slice plane: K-major core matrices of 8 rows x
// 8 BF16, 8 K-cores (1 KB) per 8-row group
__device__ __forceinline__ size_t slice_off(int64_t row, int kk) {
    return ((size_t)((row >> 3) * 8 + (kk >> 3)) * 8 + (size_t)(row & 7)) * 16 + (size_t)(kk & 7) * 2;
}

// Slices of the panel (tile column k) for the trailing rows r >= 64 (k + 1),
// in integer arithmetic on the FP64 bit patterns: eight threads per row, each
// owning 8 consecutive K values (one 16-byte core row per slice plane).
//   e_r  = (largest biased exponent of the row) - 1021, so |v| 2^-e_r < 1/2;
//   X    = round(v 2^{56 - e_r}), an integer below 2^55 (values below 2^-1022
//          are taken as 0);
//   s_p  = round(t_p / 2^{56-7p}), t_{p+1} = t_p - s_p 2^{56-7p}, t_1 = X,
// so that X = sum_p s_p 2^{56-7p} exactly with every |s_p| <= 64.
__global__ void __launch_bounds__(256) oz_slice_kernel(const double* src0, int64_t zstride, int64_t sld,
                                                       int64_t nrows, int64_t row0, int64_t rows_pad,
                                                       size_t plane_bytes, uint8_t* S, int* E) {
    const int z = blockIdx.y;
    const int tid = threadIdx.x, grp = tid & 7;  // K values 8 grp .. 8 grp + 7
    const int64_t rr = (int64_t)blockIdx.x * 32 + (tid >> 3);
    const int64_t r = row0 + rr;  // row of the slice planes
    const bool live = rr < nrows;
    long long bits[8];
    if (live) {
        const double2* src = reinterpret_cast<const double2*>(src0 + (int64_t)z * zstride + rr * sld + 8 * grp);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const double2 v = src[h];
            bits[2 * h] = __double_as_longlong(v.x);
            bits[2 * h + 1] = __double_as_longlong(v.y);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) bits[q] = 0;
    }
    int ebmax = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) ebmax = max(ebmax, (int)((bits[q] >> 52) & 0x7ff));
    // the eight threads of a row are eight consecutive lanes
    for (int o = 1; o < 8; o <<= 1) ebmax = max(ebmax, __shfl_xor_sync(0xffffffffu, ebmax, o));
    if (!live) return;
    const bool nonfinite = ebmax == 0x7ff;
    const int e = ebmax - 1021;
    uint32_t w[kSlices][4];  // BF16 pairs of the 8 values, per plane
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int eb = (int)((bits[q] >> 52) & 0x7ff);
        long long X = 0;
        if (eb != 0 && !nonfinite) {
            const long long M = (bits[q] & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
            const int sh = eb - ebmax + 2;  // <= 2
            if (sh >= 0) X = M << sh;
            else if (-sh <= 60) X = (M + (1LL << (-sh - 1))) >> (-sh);
            if (bits[q] < 0) X = -X;
        }
#pragma unroll
        for (int p = 1; p <= kSlices; ++p) {
            const int sft = 56 - 7 * p;
            const long long sp = sft > 0 ? (X + (1LL << (sft - 1))) >> sft : X;
            X -= sp << sft;
            const float f = (float)(int)sp;
            uint32_t hb;
            asm("{\n\t.reg .b16 h;\n\tcvt.rn.bf16.f32 h, %1;\n\tmov.b32 %0, {h, h};\n\t}" : "=r"(hb) : "f"(f));
            if (q & 1) w[p - 1][q >> 1] |= hb & 0xFFFF0000u;
            else w[p - 1][q >> 1] = hb & 0x0000FFFFu;
        }
    }
    uint8_t* Sz = S + (size_t)z * kSlices * plane_bytes + slice_off(r, 8 * grp);
#pragma unroll
    for (int p = 0; p < kSlices; ++p)
        *reinterpret_cast<uint4*>(Sz + (size_t)p * plane_bytes) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    // a NaN or infinity in the panel must reach the next pivot test as NaN
    if (grp == 0) E[(int64_t)z * rows_pad + r] = nonfinite ? kBadExp : e;
}

// kTrsm = false: A_ij -= A_ik A_jk^T over the trailing lower tiles (SYRK/GEMM);
// kTrsm = true:  A_ik := A_ik L_kk^{-T} for the panel tiles i > k (TRSM as a
// product with the inverse diagonal tile, whose slices sit in the plane rows
// of tile k), written instead of subtracted.
template <bool kTrsm>
__global__ void __launch_bounds__(kOzThreads, 1) oz_gemm_kernel(double* A, int nt, int k, const uint8_t* S,
                                                               size_t plane_bytes, const int* E, int* err,
                                                               int tiles_per_block, int nwork) {
    extern __shared__ __align__(1024) uint8_t oz_smem[];
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ int s_ec[T];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int rem = nt - k - 1;
    const int64_t ld = (int64_t)nt * T, rows_pad = ld + T;
    uint8_t* sA = oz_smem;
    uint8_t* sB = oz_smem + kSlices * kPlaneA;
    // work item w = (block z, super-tile): row tiles i0 = k + 1 + 2u, i0 + 1 and
    // column tile j = k + 1 + jj <= i0 + 1 (SYRK) or j = k (TRSM)
    auto decode = [&](int w, int& z, int& i0, int& j) {
        z = w / tiles_per_block;
        int u = 0, jj = w - z * tiles_per_block;
        if constexpr (kTrsm) {
            u = jj;
            jj = -1;
        } else {
            while (true) {
                const int nc = min(2 * u + 2, rem);
                if (jj < nc) break;
                jj -= nc;
                ++u;
            }
        }
        i0 = k + 1 + 2 * u;
        j = k + 1 + jj;
    };
    auto issue_loads = [&](int w) {
        int z, i0, j;
        decode(w, z, i0, j);
        const uint8_t* Sz = S + (size_t)z * kSlices * plane_bytes;
        mbar_expect_tx(&bar_load, kOzSmem);
        for (int p = 0; p < kSlices; ++p)
            bulk_g2s(sA + p * kPlaneA, Sz + (size_t)p * plane_bytes + (size_t)i0 * T * kRowBytes, kPlaneA,
                     &bar_load);
        for (int q = 0; q < kSlices; ++q)
            bulk_g2s(sB + q * kPlaneB, Sz + (size_t)q * plane_bytes + (size_t)j * T * kRowBytes, kPlaneB,
                     &bar_load);
    };

    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (tid == 0 && (int)blockIdx.x < nwork) issue_loads((int)blockIdx.x);

    // Persistent loop: the slices of the next work item are copied in while the
    // epilogue of the current one runs (shared memory is free once its MMAs are
    // done; the accumulators are free after the epilogue).
    int it = 0;
    for (int w = (int)blockIdx.x; w < nwork; w += (int)gridDim.x, ++it) {
        int z, i0, j;
        decode(w, z, i0, j);
        if (tid < T) s_ec[tid] = E[(int64_t)z * rows_pad + (int64_t)j * T + tid];
        __syncthreads();
        if (tid == 0) {
            if (mbar_wait(&bar_load, (uint32_t)(it & 1), &s_abort, err)) {
                tc_fence_after();
                constexpr uint32_t idesc = instr_desc(1, kSlabRows, T);  // BF16 x BF16 -> F32, 128 x 64
                const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
                for (int L = 2; L <= kSlices + 1; ++L) {
                    const uint32_t d = tmem + 64u * (uint32_t)(L - 2);
                    uint32_t acc = 0;
                    for (int p = max(1, L - kSlices); p <= min(kSlices, L - 1); ++p) {
                        const int q = L - p;
                        const uint32_t ap = a0 + (uint32_t)(p - 1) * kPlaneA, bq = b0 + (uint32_t)(q - 1) * kPlaneB;
#pragma unroll
                        for (int ks = 0; ks < T / 16; ++ks) {
                            mma_ss(d, smem_desc(ap + ks * 256, 128, 1024), smem_desc(bq + ks * 256, 128, 1024),
                                   idesc, acc);
                            acc = 1;
                        }
                    }
                }
                tc_commit(&bar_mma);
            }
        }
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_mma, (uint32_t)(it & 1), &s_abort, err));
        if (ok) tc_fence_after();
        // the shared slices are consumed: fetch the next work item's
        if (tid == 0 && ok && w + (int)gridDim.x < nwork) issue_loads(w + (int)gridDim.x);

        // epilogue: warp v owns tensor-memory lanes (rows) 32 (v % 4) .. + 31 and
        // columns 32 (v / 4) .. + 31 of the super-tile
        const int rl = 32 * (warp & 3) + (tid & 31);
        const int64_t r = (int64_t)i0 * T + rl;
        const int rtile = i0 + rl / T;
        const bool live = ok && rtile < nt && (kTrsm || j <= rtile);
        const int er = live ? E[(int64_t)z * rows_pad + r] : 0;
        double* Crow = A + (int64_t)z * ld * ld + r * ld + (int64_t)j * T;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        // exact conversions: an FP32 integer below 2^22 through the FP32 mantissa,
        // a 64-bit integer below 2^51 through the FP64 mantissa
        constexpr float kMagicF = 12582912.0f;                  // 1.5 * 2^23
        constexpr long long kMagicDBits = 0x4338000000000000LL;  // 1.5 * 2^52
        constexpr double kMagicD = 6755399441055744.0;
#pragma unroll 1
        for (int c0 = 32 * (warp >> 2); c0 < 32 * (warp >> 2) + 32; c0 += 16) {
            long long H[16], Lo[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) H[c] = Lo[c] = 0;
#pragma unroll
            for (int L = 2; L <= kSlices + 1; ++L) {
                uint32_t v[16];
                if (ok) {
                    tmem_ld16(tmem + lane_base + 64u * (uint32_t)(L - 2) + (uint32_t)c0, v);
                    tmem_wait_ld();
                } else {
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] = 0u;
                }
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const long long iv =
                        (long long)(__float_as_int(__uint_as_float(v[c]) + kMagicF) - __float_as_int(kMagicF));
                    if (L <= 5) H[c] = H[c] * 128 + iv;
                    else Lo[c] = Lo[c] * 128 + iv;
                }
            }
            if (live) {
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const double hd = __longlong_as_double(kMagicDBits + H[c]) - kMagicD;
                    const double ld_ = __longlong_as_double(kMagicDBits + Lo[c]) - kMagicD;
                    const double t = fma(ld_, 0x1p-28, hd);
                    const int ec = s_ec[c0 + c];
                    const int e = er + ec - 35;
                    double scale;
                    if (e >= -1022 && e <= 1023) scale = __longlong_as_double((long long)(e + 1023) << 52);
                    else scale = ldexp(1.0, max(-1074, min(1023, e)));
                    const double nv = kTrsm ? t * scale : fma(-t, scale, Crow[c0 + c]);
                    Crow[c0 + c] = (er == kBadExp || ec == kBadExp) ? __longlong_as_double(0x7ff8000000000000LL) : nv;
                }
            }
        }
        // every accumulator has been read before the next MMAs overwrite them
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (s_abort) break;
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        if (s_abort) {
            // a wait gave up: let copies and MMAs still in flight land first
            const long long t0 = clock64();
            while (clock64() - t0 < 4000000LL) {
            }
        }
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// persistent grid: one CTA per SM (the slice planes fill shared memory)
int sm_count() {
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            sms = v;
        else
            sms = 148;
        cudaGetLastError();
    }
    return sms;
}

}  // namespace

size_t oz_plane_bytes(int nt) { return (size_t)((int64_t)nt * T + T) * kRowBytes; }
size_t oz_slice_bytes(int nt) { return kSlices * oz_plane_bytes(nt); }
size_t oz_expo_ints(int nt) { return (size_t)((int64_t)nt * T + T); }

cudaError_t launch_oz_update(double* A, int nt, int k, int g, uint8_t* S, int* E, int* err, cudaStream_t st,
                             int64_t* launches) {
    const int rem = nt - k - 1;
    if (rem <= 0) return cudaSuccess;
    static_assert(kOzSmem + 1024 <= 227 * 1024, "shared memory");
    cudaError_t e =
        cudaFuncSetAttribute(oz_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
    if (e != cudaSuccess) return e;
    const size_t pb = oz_plane_bytes(nt);
    const int64_t ld = (int64_t)nt * T;
    const int64_t rows = (int64_t)rem * T;
    oz_slice_kernel<<<dim3((unsigned)((rows + 31) / 32), (unsigned)g), 256, 0, st>>>(
        A + (int64_t)(k + 1) * T * ld + (int64_t)k * T, ld * ld, ld, rows, (int64_t)(k + 1) * T, ld + T, pb, S, E);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int tiles = 0;
    for (int u = 0; 2 * u < rem; ++u) tiles += std::min(2 * u + 2, rem);
    const int nwork = tiles * g;
    oz_gemm_kernel<false><<<(unsigned)std::min(nwork, sm_count()), kOzThreads, kOzSmem, st>>>(A, nt, k, S, pb, E, err,
                                                                                            tiles, nwork);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_oz_trsm(double* A, const double* Dinv, int nt, int k, int g, uint8_t* S, int* E, int* err,
                           cudaStream_t st, int64_t* launches) {
    const int rem = nt - k - 1;
    if (rem <= 0) return cudaSuccess;
    cudaError_t e =
        cudaFuncSetAttribute(oz_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
    if (e != cudaSuccess) return e;
    const size_t pb = oz_plane_bytes(nt);
    const int64_t ld = (int64_t)nt * T;
    const int64_t rows = (int64_t)rem * T;
    // the panel below the diagonal tile, and L_kk^{-1} into the plane rows of tile k
    oz_slice_kernel<<<dim3((unsigned)((rows + 31) / 32), (unsigned)g), 256, 0, st>>>(
        A + (int64_t)(k + 1) * T * ld + (int64_t)k * T, ld * ld, ld, rows, (int64_t)(k + 1) * T, ld + T, pb, S, E);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    oz_slice_kernel<<<dim3(T / 32, (unsigned)g), 256, 0, st>>>(Dinv + (int64_t)k * T * T, (int64_t)nt * T * T, T,
                                                                T, (int64_t)k * T, ld + T, pb, S, E);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int tiles = (rem + 1) / 2, nwork = tiles * g;
    oz_gemm_kernel<true><<<(unsigned)std::min(nwork, sm_count()), kOzThreads, kOzSmem, st>>>(A, nt, k, S, pb, E, err,
                                                                                           tiles, nwork);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

}  // namespace ap
