// Tensor-core (tcgen05) form of the fused AP residual update (Eq. text_update_of_r)
// with the Gauss-Southwell epilogue (Eq. approximate_gauss_southwell).
//
// Per 128-row tile of R and per 128-column chunk of the selected block I:
//   1. S_ij = |x_s,i - x_s,j|^2 = t_ij on the tensor cores as one product of
//      [x_hi | x_hi | x_lo | a_hi | a_lo | 1 | 1] and
//      [-2x'_hi | -2x'_lo | -2x'_hi | 1 | 1 | a'_hi | a'_lo] (a = |x_s|^2, every
//      value split into an FP16 hi/lo pair; the three cross products of the
//      pairs are laid out along K, so K = 3d + 4 rounded up to 16 and d <= 4
//      needs a single MMA), FP32 accumulation in tensor memory;
//   2. twenty transform warps load t from tensor memory, evaluate phi on the
//      SFU and write P = phi back as a BF16 hi/lo pair, in place: every 16
//      FP32 columns of S become 8 columns of P_hi followed by 8 of P_lo;
//   3. acc += P Delta^T on the tensor cores with P read from tensor memory and
//      Delta^T (BF16 hi/lo, staged per step) from shared memory: the three
//      products hi*hi + hi*lo + lo*hi carry about 16 bits.
// After the last chunk the accumulator (128 x C FP32) leaves tensor memory and
// R_i -= s acc_i + sigma^2 Delta_i (index diagonal), with the block norms of the
// new R written per tile for the ticketed last-CTA selection.
//
// Warp roles: warps 0-19 transform (warp w owns TMEM lanes 32 (w % 4).. and
// takes 32-column work items of the chunks round-robin with the other four
// warps of its lane quarter; five transform warps per scheduler hide the SFU
// and tensor-memory latencies); warp 20 issues the distance MMAs, warp 21 the
// contraction MMAs and warp 22 (lane 0) the bulk copies, so that no issuer
// waits behind another one's barriers.  The MMA issuers run their loops on the
// whole warp, with warp-uniform addresses and descriptors, and issue from one
// elected lane: a loop in a single lane of a diverged warp paid some 70-80
// cycles per MMA and made the contraction issuer the bottleneck.  The hi*hi
// and hi*lo products of the contraction are one MMA of width 2C (Delta_hi and
// Delta_lo stacked), lo*hi a second one into its own accumulator; the three
// partial sums are added in the epilogue.  S/P live in a ring of three
// tensor-memory buffers (a buffer is reused once the contraction that read its
// P has completed), operands in a ring of shared-memory stages; everything is
// synchronised by mbarriers, and every wait is bounded in time and reports a
// timeout through the error flag instead of hanging.
//
// Work split: the (tile, chunk) pairs of a step, in tile-major order, are cut
// into one equal contiguous range per persistent CTA (instead of whole tiles,
// which leave the last wave partly idle: 2048 tiles on 152 SMs are 13.5 each).
// A tile that straddles two ranges is accumulated in two parts; both go to a
// boundary slot in global memory and the second CTA to arrive (an atomic
// ticket, no waiting) adds them in a fixed order and updates R.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kmv_fp32.cuh"
#include "tcgen05.cuh"

namespace ap {
namespace tc {

constexpr int kRows = 128;
constexpr int kChunk = 128;  // columns of the block per chunk
constexpr int kStages = 4;
constexpr int kBufs = 3;     // S/P tensor-memory buffers
constexpr int kColsPerWarp = 32;                   // columns of a chunk per work item (two 16-column units)
constexpr int kUnits = kColsPerWarp / 16;          // 16-column units per work item
constexpr int kGroups = kChunk / kColsPerWarp;     // work items (column groups) of a chunk per lane quarter
constexpr int kSlots = 5;                          // transform warps per lane quarter
constexpr int kXformWarps = 4 * kSlots;
constexpr int kLoadWarp = kXformWarps;       // distance MMAs (also owns the tensor memory)
constexpr int kMmaWarp = kXformWarps + 1;    // contraction MMAs
constexpr int kCopyWarp = kXformWarps + 2;   // bulk copies of the operand stages
constexpr int kThreads = (kXformWarps + 3) * 32;
static_assert(2 * kGroups >= kSlots, "a transform warp has a work item in one of any two consecutive chunks");
constexpr int kEpiSets = 4;  // named barriers / shared buffers of tile epilogues in flight
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColAcc = kBufs * kChunk;  // three accumulators (hi*hi, hi*lo, lo*hi), C columns each
static_assert(kColAcc + 3 * 32 <= kTmemCols, "tensor memory budget");
}  // namespace tc

// K of the distance product for d <= 30 (the tensor-core forms' limit): 3d + 4
// rounded up to 16; shared memory is sized for it at the largest d.
constexpr int kTcMaxKdp = 96;

namespace tc {
// phi from the tensor-core distance t.  RBF operands carry the FP32 path's
// scaling (t = r^2 log2(e) / 2, phi = 2^-t).  Matern operands are additionally
// scaled by log2(e), so sqrt(t) = u log2(e) with u = sqrt(3 or 5) r, which puts
// e^-u on the SFU without a multiply; the polynomial takes the 1/log2(e) powers.
constexpr float kInvL = 0.69314718055994531f;                 // 1 / log2(e)
constexpr float kInvL2Third = 0.69314718055994531f * 0.69314718055994531f / 3.0f;

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_elem), "f"(lo_elem));
    return r;
}

__device__ __forceinline__ float bf16_lo_to_f32(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi_to_f32(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Paired FP32 arithmetic (one instruction for two lanes of a float2, each lane
// rounded exactly as the scalar operation).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// phi of two distances at once: the SFU work per lane, the Matern polynomial in
// scalar FMAs (their constants are immediate operands; the paired form needs
// them in register pairs and measured slower).
template <int KERN>
__device__ __forceinline__ float2 phi_tc2(float t0, float t1) {
    if constexpr (KERN == AP_RBF) {
        return make_float2(ex2_approx(-t0), ex2_approx(-t1));
    } else {
        const float u0 = sqrt_approx(fabsf(t0)), u1 = sqrt_approx(fabsf(t1));
        const float e0 = ex2_approx(-u0), e1 = ex2_approx(-u1);
        float p0, p1;
        if constexpr (KERN == AP_MATERN32) {
            p0 = fmaf(u0, kInvL, 1.0f);
            p1 = fmaf(u1, kInvL, 1.0f);
        } else {
            p0 = fmaf(fmaf(u0, kInvL2Third, kInvL), u0, 1.0f);
            p1 = fmaf(fmaf(u1, kInvL2Third, kInvL), u1, 1.0f);
        }
        return make_float2(p0 * e0, p1 * e1);
    }
}

}  // namespace tc

// Spinning wait (no suspension: the phase is picked up as soon as it completes),
// bounded like mbar_wait; the contraction issuer's wait for P in the RBF form.
__device__ __forceinline__ bool mbar_wait_spin(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err_flag,
                                               long long limit) {
    if (tc::mbar_test_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t it = 1;; ++it) {
        if (tc::mbar_test_wait(bar, parity)) return true;
        if ((it & 31u) == 0) {
            if (*abort_flag) return false;
            if (clock64() - t0 > limit) {
                *abort_flag = 1;
                atomicExch(err_flag, 1);
                return false;
            }
        }
    }
}

// -------------------------------------------------------------- kernel params
struct TcParams {
    const uint8_t* XA;     // row operand tiles: ntiles x (128 x kdp fp16)
    const uint8_t* XB;     // column operand chunks: m x cpb x (128 x kdp fp16)
    int kdp;               // K of the distance product (multiple of 16)
    const uint8_t* DT;     // Delta^T chunks of this step: cpb x (2 x C x 128 bf16)
    const float* Delta;    // b x C FP32 (noise diagonal)
    float* R;              // n x C
    int64_t n, b;
    int cpb;               // chunks per block
    float s, noise;
    const int* sel;
    int* err;              // timeout flag
    long long wait_cycles; // bound of every mbarrier wait, in SM clock cycles
    float* scr;            // gridDim.x x 2 x 128 x C: partial accumulators of the tiles two CTAs share
    int* tick;             // gridDim.x arrival counters of those tiles (0 between launches)
    EpiParams epi;         // tiles of 128 rows aligned to blocks (tiles_per_seg = ceil(b / 128))
};

// What a tile epilogue needs from the kernel: parameters by value and the
// CTA's shared barriers and buffers.
struct TcEpiArgs {
    float* R;
    const float* Delta;
    float* scr;
    int* tick;
    int* err;
    long long wait_cycles;
    float s, noise;
    int64_t n, col0, ncols;
    int64_t seg, tiles_per_seg;
    int64_t ntiles;  // row tiles of the step (size of part_norm)
    int flags;
    double* part_norm;
    double* part_col;
    uint64_t* bar_acc_full;  // [kEpiSets]
    uint64_t* bar_acc_free;
    volatile int* abort_flag;
    int* fin;           // [kEpiSets]
    double* red;        // [kEpiSets][4]
    double* colred;     // [kEpiSets][4][C]
    uint32_t tmem_acc;  // first accumulator column (lane 0)
};

// Epilogue of one row tile (segment sg of this CTA), run by four warps, one per
// lane quarter, one row per thread.  A whole tile updates R from the
// accumulators; a tile shared with a neighbouring CTA first stores its part
// (part 0: chunks from the tile's start, part 1: the rest) in the boundary
// slot, and the second CTA to arrive updates R from part 0 + part 1, in that
// order whichever arrives last.  Every path passes the same named barriers so
// that a failed wait cannot strand the others.  Out of line: it runs once per
// tile and its registers stay out of the transform loop.  Returns ok.
template <int C>
__device__ __noinline__ bool tc_tile_epilogue(const TcEpiArgs a, int quarter, int sg, int64_t tile, bool whole,
                                              int part, bool ok) {
    using namespace tc;
    const int lane = threadIdx.x & 31;
    const int es = sg % kEpiSets;
    const int bar_id = 1 + es;
    const bool elead = quarter == 0 && lane == 0;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    // segment sg completes phase sg / kEpiSets of its set's barrier
    if (ok)
        ok = __all_sync(0xffffffffu, mbar_wait(a.bar_acc_full + es, (uint32_t)((sg / kEpiSets) & 1), a.abort_flag,
                                              a.err, a.wait_cycles));
    if (ok) tc_fence_after();
    const int64_t segi = tile / a.tiles_per_seg;
    const int64_t seg_lo = segi * a.seg;
    const int64_t seg_hi = min(seg_lo + a.seg, a.n);
    const int row = quarter * 32 + lane;
    const int64_t i = seg_lo + (tile % a.tiles_per_seg) * kRows + row;
    const bool diag = i >= a.col0 && i < a.col0 + a.ncols;
    // the three partial products (hi*hi, hi*lo, lo*hi) of 16 columns
    auto acc16 = [&](int c0, float (&a16)[16]) {
        uint32_t r[16];
        tmem_ld16(a.tmem_acc + lane_base + c0, r);
        tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) a16[k] = __uint_as_float(r[k]);
        tmem_ld16(a.tmem_acc + lane_base + C + c0, r);
        tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) a16[k] += __uint_as_float(r[k]);
        tmem_ld16(a.tmem_acc + lane_base + 2 * C + c0, r);
        tmem_wait_ld();
#pragma unroll
        for (int k = 0; k < 16; ++k) a16[k] += __uint_as_float(r[k]);
    };
    bool apply = whole;
    const int64_t bnd = part == 0 ? (int64_t)blockIdx.x : (int64_t)blockIdx.x - 1;
    float* scr0 = a.scr + ((bnd * 2 + 0) * kRows + row) * C;
    float* scr1 = a.scr + ((bnd * 2 + 1) * kRows + row) * C;
    if (!whole) {
        if (ok) {
            float* mine = part == 0 ? scr0 : scr1;
            if (!AP_CHK(bnd >= 0 && bnd < (int64_t)gridDim.x)) mine = nullptr;
#pragma unroll 1
            for (int c0 = 0; c0 < C; c0 += 16) {
                float a16[16];
                acc16(c0, a16);
#pragma unroll
                for (int k = 0; k < 16; k += 4)
                    if (mine)
                        __stcg(reinterpret_cast<float4*>(mine + c0 + k),
                               make_float4(a16[k], a16[k + 1], a16[k + 2], a16[k + 3]));
            }
            tc_fence_before();
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(a.bar_acc_free);
        __threadfence();
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        if (elead) {
            int fin = 0;
            if (ok) {
                fin = AP_CHK(bnd >= 0 && bnd < (int64_t)gridDim.x) && atomicAdd(&a.tick[bnd], 1) == 1;
                if (fin) a.tick[bnd] = 0;  // both parts are in: ready for the next launch
                __threadfence();
            }
            a.fin[es] = fin;
        }
        asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
        apply = a.fin[es] != 0;
    }
    const bool live = ok && apply && i < seg_hi && AP_CHK(i < a.n) &&
                      (whole || AP_CHK(bnd >= 0 && bnd < (int64_t)gridDim.x));
    // squares are summed in FP32 within a thread and a warp (at most 32 terms
    // each, relative error below 2e-6) and in FP64 beyond: FP64 arithmetic is
    // scarce on this part
    float sqf = 0.0f;
    double* colred = a.colred + (size_t)es * 4 * C;
    // 16 columns at a time: the accumulated product, R update, norms
#pragma unroll 1
    for (int c0 = 0; c0 < C; c0 += 16) {
        float a16[16];
        if (ok && whole) {
            acc16(c0, a16);
        } else if (live) {
#pragma unroll
            for (int k = 0; k < 16; ++k) a16[k] = __ldcg(scr0 + c0 + k) + __ldcg(scr1 + c0 + k);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float v = 0.0f;
            if (live) {
                const int c = c0 + k;
                v = fmaf(-a.s, a16[k], a.R[i * C + c]);
                if (diag && AP_CHK(i - a.col0 < a.ncols)) v = fmaf(-a.noise, a.Delta[(i - a.col0) * C + c], v);
                a.R[i * C + c] = v;
                sqf = fmaf(v, v, sqf);
            }
            if (apply && (a.flags & kEpiColNorms)) {
                float w = v * v;
                for (int off = 16; off > 0; off >>= 1) w += __shfl_down_sync(0xffffffffu, w, off);
                if (lane == 0) colred[quarter * C + c0 + k] = (double)w;
            }
        }
    }
    if (whole) {
        if (ok) tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(a.bar_acc_free);
    }
    double sq = sqf;
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
    if (lane == 0) a.red[es * 4 + quarter] = sq;
    asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
    if (elead && apply && AP_CHK(tile >= 0 && tile < a.ntiles)) {
        const double* rd = a.red + es * 4;
        a.part_norm[tile] = rd[0] + rd[1] + rd[2] + rd[3];
        if (a.flags & kEpiColNorms)
            for (int c = 0; c < C; ++c) a.part_col[tile * C + c] = colred[c] + colred[C + c] + colred[2 * C + c] + colred[3 * C + c];
    }
    asm volatile("bar.sync %0, 128;" ::"r"(bar_id) : "memory");
    return ok;
}

template <int KERN, int C>
__global__ void __launch_bounds__(tc::kThreads, 1) kmv_tc_kernel(const TcParams p) {
    using namespace tc;
    const uint32_t kXaBytes = (uint32_t)(kRows * p.kdp * 2);
    const uint32_t kXbBytes = (uint32_t)(kChunk * p.kdp * 2);
    constexpr uint32_t kDtBytes = 2u * C * kChunk * 2u;   // hi + lo
    const uint32_t kStageBytes = kXbBytes + kDtBytes;
    const int KSTEPS_D = p.kdp / 16;
    constexpr int KSTEPS_C = kChunk / 16;
    const uint32_t kSboX = (uint32_t)(p.kdp / 8) * 128;  // 8-row groups of the X operands
    constexpr uint32_t kSboD = (kChunk / 8) * 128;       // 8-row groups of Delta^T

    extern __shared__ __align__(1024) uint8_t tc_smem[];
    uint8_t* s_xa = tc_smem;                         // 2 buffers
    uint8_t* s_stage = tc_smem + 2 * kXaBytes;       // kStages buffers
    __shared__ __align__(8) uint64_t bar_stage_full[kStages], bar_stage_empty[kStages];
    __shared__ __align__(8) uint64_t bar_xa_full[2], bar_xa_empty[2];
    // per S/P buffer: S written (distance MMAs), P of one column group written
    // (its four transform warps), P consumed (contraction MMAs)
    __shared__ __align__(8) uint64_t bar_s_full[kBufs], bar_p_full[kBufs][kGroups], bar_buf_free[kBufs];
    // accumulators of a tile complete (one barrier per epilogue set: the tile
    // epilogues of consecutive segments run on different warps, and a segment
    // may be a single chunk, so a warp group can reach its wait before the
    // previous segment's product has completed) / read by the epilogue
    __shared__ __align__(8) uint64_t bar_acc_full[kEpiSets], bar_acc_free;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ double red_d[32];
    __shared__ int red_i[32];
    // tile epilogues: consecutive tiles may overlap in time (different warps),
    // so each takes its own set of reduction buffers and named barrier
    __shared__ double e_red[kEpiSets][4];
    __shared__ double s_colred[kEpiSets][4][C];
    __shared__ int s_last;
    __shared__ int s_fin[kEpiSets];  // this CTA completes a shared tile

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const EpiParams& e = p.epi;

    const int I = *p.sel;
    const int64_t col0 = (int64_t)I * p.b;
    const int64_t ncols = min(p.b, p.n - col0);
    const int nq = (int)((ncols + kChunk - 1) / kChunk);
    const int64_t ntiles = e.ntiles;
    // Work units are (tile, chunk) pairs in tile-major order, split into equal
    // contiguous ranges, one per CTA.  With gridDim.x <= ntiles every range holds
    // at least nq units, so a tile is shared by at most two CTAs (the end of one
    // range and the start of the next); their partial accumulators meet in a
    // boundary slot and the second to arrive updates R.  A "segment" is the part
    // of one tile inside this CTA's range.
    const int64_t U = ntiles * nq;
    const int64_t u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
    const int64_t total = u1 - u0;

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&bar_stage_full[i], 1);
            mbar_init(&bar_stage_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_xa_full[i], 1);
            mbar_init(&bar_xa_empty[i], 1);
        }
        for (int i = 0; i < kBufs; ++i) {
            mbar_init(&bar_s_full[i], 1);
            for (int gq = 0; gq < kGroups; ++gq) mbar_init(&bar_p_full[i][gq], 4);
            mbar_init(&bar_buf_free[i], 1);
        }
        for (int i = 0; i < kEpiSets; ++i) mbar_init(&bar_acc_full[i], 1);
        mbar_init(&bar_acc_free, 4);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kLoadWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == kCopyWarp) {
        // ------------------------------------------------ bulk-copy issuer
        if (lane == 0 && total > 0) {
            // a bound shorter than the default (tests of the timeout path) is
            // enforced here with non-blocking probes: the copy issuer runs ahead
            // of the pipeline, so its waits are the ones that run out
            const bool strict = p.wait_cycles < kWaitCycles;
            auto copy_wait = [&](uint64_t* bar, uint32_t parity) -> bool {
                return strict ? mbar_wait_strict(bar, parity, &s_abort, p.err, p.wait_cycles)
                              : mbar_wait(bar, parity, &s_abort, p.err, p.wait_cycles);
            };
            auto issue_xa = [&](int64_t sg, int64_t tile) -> bool {
                const int xb = (int)(sg & 1);
                const int64_t u = sg >> 1;
                if (u >= 1 && !copy_wait(&bar_xa_empty[xb], (uint32_t)((u - 1) & 1))) return false;
                // (an index that fails its check arrives with no bytes: nothing is copied)
                const bool in = AP_CHK(tile >= 0 && tile < e.ntiles);
                mbar_expect_tx(&bar_xa_full[xb], in ? kXaBytes : 0u);
                if (in) bulk_g2s(s_xa + (size_t)xb * kXaBytes, p.XA + (size_t)tile * kXaBytes, kXaBytes, &bar_xa_full[xb]);
                return true;
            };
            int64_t tile = u0 / nq, sg = 0;
            int q = (int)(u0 % nq);
            const int64_t last_tile = (u1 - 1) / nq;
            bool ok = issue_xa(0, tile);
            for (int64_t i = 0; i < total && ok; ++i) {
                if ((i == 0 || q == 0) && tile < last_tile) ok = issue_xa(sg + 1, tile + 1);
                const int s = (int)(i % kStages);
                const int64_t u = i / kStages;
                if (ok && u >= 1) ok = copy_wait(&bar_stage_empty[s], (uint32_t)((u - 1) & 1));
                if (!ok) break;
                uint8_t* dst = s_stage + (size_t)s * kStageBytes;
                const bool in = AP_CHK(I >= 0 && I < e.m && q >= 0 && q < p.cpb);
                mbar_expect_tx(&bar_stage_full[s], in ? kStageBytes : 0u);
                if (in) {
                    bulk_g2s(dst, p.XB + ((size_t)I * p.cpb + q) * kXbBytes, kXbBytes, &bar_stage_full[s]);
                    bulk_g2s(dst + kXbBytes, p.DT + (size_t)q * kDtBytes, kDtBytes, &bar_stage_full[s]);
                }
                if (++q == nq) {
                    q = 0;
                    ++tile;
                    ++sg;
                }
            }
        }
    } else if (warp == kLoadWarp) {
        // ------------------------------------------------ distance MMA issuer
        // The whole warp runs the loop (warp-uniform addresses and descriptors);
        // one elected lane issues the MMAs and their commits.
        if (total > 0) {
            constexpr uint32_t idesc_d = instr_desc(0, kRows, kChunk);  // F16 x F16 -> F32, 128 x 128
            const bool leader = elect_one();
            bool ok = true;
            int64_t sg = -1;
            int q = (int)(u0 % nq), xb = 0;
            uint64_t da = 0;
            const uint64_t db0 = smem_desc(smem_u32(s_stage), 128, kSboX);
            for (int64_t g = 0; g < total && ok; ++g) {
                if (g == 0 || q == 0) {
                    ++sg;
                    xb = (int)(sg & 1);
                    ok = __all_sync(0xffffffffu,
                                    mbar_wait(&bar_xa_full[xb], (uint32_t)((sg >> 1) & 1), &s_abort, p.err, p.wait_cycles));
                    da = smem_desc(smem_u32(s_xa + (size_t)xb * kXaBytes), 128, kSboX);
                    if (!ok) break;
                }
                const int s = (int)(g % kStages);
                const int buf = (int)(g % kBufs);
                const int64_t use = g / kBufs;
                ok = __all_sync(0xffffffffu,
                                mbar_wait(&bar_stage_full[s], (uint32_t)((g / kStages) & 1), &s_abort, p.err, p.wait_cycles));
                if (ok && use >= 1)
                    ok = __all_sync(0xffffffffu, mbar_wait(&bar_buf_free[buf], (uint32_t)((use - 1) & 1), &s_abort, p.err,
                                                          p.wait_cycles));
                if (!ok) break;
                tc_fence_after();
                // descriptor address fields advance by 16-byte units: stage s, K-step ks (256 B)
                const uint64_t db = db0 + (uint64_t)((s * kStageBytes) >> 4);
                const uint32_t dS = tmem + (uint32_t)(kChunk * buf);
                if (leader) {
                    for (int ks = 0; ks < KSTEPS_D; ++ks)
                        mma_ss(dS, da + (uint64_t)(ks * 16), db + (uint64_t)(ks * 16), idesc_d, ks > 0 ? 1u : 0u);
                    tc_commit(&bar_s_full[buf]);
                    if (g == total - 1 || q == nq - 1) tc_commit(&bar_xa_empty[xb]);
                }
                __syncwarp();
                if (++q == nq) q = 0;
            }
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------ contraction MMA issuer
        // (whole warp in the loop, elected lane issuing, as above)
        if (total > 0) {
            // BF16 x BF16 -> F32: 128 x 2C (P_hi against [Delta_hi; Delta_lo]) and 128 x C
            constexpr uint32_t idesc_c2 = instr_desc(1, kRows, 2 * C);
            constexpr uint32_t idesc_c = instr_desc(1, kRows, C);
            const bool leader = elect_one();
            const uint64_t dt0 = smem_desc(smem_u32(s_stage + kXbBytes), 128, kSboD);
            const uint32_t a01 = tmem + kColAcc, a2 = a01 + 2 * C;
            bool ok = true;
            int64_t sg = -1;
            int q = (int)(u0 % nq);
            for (int64_t g = 0; g < total && ok; ++g) {
                const bool first = g == 0 || q == 0;
                const int buf = (int)(g % kBufs);
                const int s = (int)(g % kStages);
                const uint32_t ph = (uint32_t)((g / kBufs) & 1);
                if (first && ++sg >= 1)
                    ok = __all_sync(0xffffffffu,
                                    mbar_wait(&bar_acc_free, (uint32_t)((sg - 1) & 1), &s_abort, p.err, p.wait_cycles));
                if (!ok) break;
                // Delta^T of the stage: C rows of Delta_hi, then C rows of Delta_lo
                // (consecutive 8-row groups), so one N = 2C product gives hi*hi
                // and hi*lo side by side in accumulator columns [0, 2C)
                const uint64_t dth = dt0 + (uint64_t)((s * kStageBytes) >> 4);
                const uint32_t pb = tmem + (uint32_t)(kChunk * buf);
                // K-step ks: 16 BF16 values of P = 8 columns of P_hi at 16 ks and 8
                // of P_lo at 16 ks + 8; two 16-byte core columns of Delta^T (core
                // columns 128 B apart).  The K-steps of a column group start as
                // soon as its four transform warps have written their P.
#pragma unroll
                for (int ks = 0; ks < KSTEPS_C; ++ks) {
                    if (ks % kUnits == 0) {
                        // RBF (one SFU operation per entry, short chunk periods) picks P
                        // up by spinning; for the Matern kernels the spin's issue slots
                        // cost the transform warps of this scheduler more than it saves
                        uint64_t* pf = &bar_p_full[buf][ks / kUnits];
                        const bool got = KERN == AP_RBF ? mbar_wait_spin(pf, ph, &s_abort, p.err, p.wait_cycles)
                                                        : mbar_wait(pf, ph, &s_abort, p.err, p.wait_cycles);
                        ok = __all_sync(0xffffffffu, got);
                        if (!ok) break;
                        tc_fence_after();
                    }
                    const uint32_t acc = (first && ks == 0) ? 0u : 1u;
                    const uint64_t bd = dth + (uint64_t)(ks * 16);
                    const uint32_t pH = pb + 16u * ks, pL = pH + 8u;
                    if (leader) {
                        mma_ts(a01, pH, bd, idesc_c2, acc);
                        mma_ts(a2, pL, bd, idesc_c, acc);
                    }
                }
                if (!ok) break;
                if (leader) {
                    tc_commit(&bar_buf_free[buf]);
                    tc_commit(&bar_stage_empty[s]);
                    if (g == total - 1 || q == nq - 1) tc_commit(&bar_acc_full[sg % kEpiSets]);
                }
                __syncwarp();
                if (++q == nq) q = 0;
            }
        }
    } else {
        // ------------------------------------------------ transform warps
        // A chunk is 4 work items of 32 columns per lane quarter; the 5
        // transform warps of a quarter (warp = 4 slot + quarter, which fixes its
        // TMEM lanes) take the items of the CTA's chunk sequence round-robin (item
        // 4 c + g to slot (4 c + g) mod 5), each item as two 16-column units (16
        // entries per thread each) loaded together and transformed interleaved.
        // Every warp has an item in one of any two consecutive chunks, so no S/P
        // buffer can run two phases ahead of it.  The tile epilogue of segment sg
        // runs on the four warps of slot sg mod 5, after they finished their items
        // up to the segment's last chunk.
        const int quarter = warp & 3, slot = warp >> 2;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        bool ok = total > 0;
        // Chunk c of this CTA is pair u0 + c: tile (u0 + c) / nq, chunk (u0 + c) % nq
        // of the block.  Segment sg = the chunks of tile tile0 + sg.  Per-item
        // bookkeeping is kept in incremental 32-bit counters (no divisions in the
        // loop): the item's chunk c and group, S/P buffer c mod 3 and its phase.
        const int ntot = (int)total;
        const int64_t tile0 = nq > 0 ? u0 / nq : 0;
        const int nseg = ntot > 0 ? (int)((u1 - 1) / nq - tile0 + 1) : 0;
        const int qa = nq > 0 ? (int)(u0 % nq) : 0;  // chunk index of the CTA's first pair within its tile
        auto seg_last = [&](int sg) -> int {  // last chunk of segment sg
            return min(ntot - 1, (sg + 1) * nq - 1 - qa);
        };
        // the epilogue's arguments are assembled at each call (from kernel
        // parameters and shared addresses), so that none of them stays live
        // across the transform loop
        auto run_epilogue = [&](int sg) {
            TcEpiArgs ea;
            ea.R = p.R;
            ea.Delta = p.Delta;
            ea.scr = p.scr;
            ea.tick = p.tick;
            ea.err = p.err;
            ea.wait_cycles = p.wait_cycles;
            ea.s = p.s;
            ea.noise = p.noise;
            ea.n = p.n;
            ea.col0 = col0;
            ea.ncols = ncols;
            ea.seg = e.seg;
            ea.tiles_per_seg = e.tiles_per_seg;
            ea.ntiles = e.ntiles;
            ea.flags = e.flags;
            ea.part_norm = e.part_norm;
            ea.part_col = e.part_col;
            ea.bar_acc_full = bar_acc_full;
            ea.bar_acc_free = &bar_acc_free;
            ea.abort_flag = &s_abort;
            ea.fin = s_fin;
            ea.red = &e_red[0][0];
            ea.colred = &s_colred[0][0][0];
            ea.tmem_acc = tmem + kColAcc;
            const int c_first = max(0, sg * nq - qa);
            const int q_first = (qa + c_first) % nq, q_last = (qa + seg_last(sg)) % nq;
            ok = tc_tile_epilogue<C>(ea, quarter, sg, tile0 + sg, q_first == 0 && q_last == nq - 1, q_first == 0 ? 0 : 1,
                                     ok);
        };
        int sg_next = 0, sg_end = nseg > 0 ? seg_last(0) : -1;
        int c_waited = -1;
        static_assert(kUnits == 2, "two units per work item");
        static_assert(kSlots < 2 * kGroups, "an item advances at most two chunks");
        int c = slot / kGroups, group = slot % kGroups;
        int buf = c % kBufs;
        uint32_t phase = (uint32_t)((c / kBufs) & 1);
        while (c < ntot) {
            // epilogues of the segments that ended before this chunk
            while (sg_next < nseg && c > sg_end) {
                if (sg_next % kSlots == slot) run_epilogue(sg_next);
                if (++sg_next < nseg) sg_end = seg_last(sg_next);
            }
            if (c != c_waited) {
                if (ok)
                    ok = __all_sync(0xffffffffu, mbar_wait(&bar_s_full[buf], phase, &s_abort, p.err, p.wait_cycles));
                if (ok) tc_fence_after();
                c_waited = c;
            }
            // columns of unit h of the item: S there is replaced by [P_hi | P_lo]
            const uint32_t addr0 = tmem + lane_base + (uint32_t)(kChunk * buf + kColsPerWarp * group);
            uint32_t ta[16], tb[16];
            if (ok) {
                tmem_ld16(addr0, ta);
                tmem_ld16(addr0 + 16, tb);
                tmem_wait_ld();
            }
            uint32_t pa[16], pb[16];  // [P_hi words | P_lo words] of each unit
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float2 v = phi_tc2<KERN>(__uint_as_float(ta[2 * k]), __uint_as_float(ta[2 * k + 1]));
                const float2 w = phi_tc2<KERN>(__uint_as_float(tb[2 * k]), __uint_as_float(tb[2 * k + 1]));
                const uint32_t hv = pack_bf16(v.x, v.y), hw = pack_bf16(w.x, w.y);
                pa[k] = hv;
                pb[k] = hw;
                const float2 lv = sub2(v, make_float2(bf16_lo_to_f32(hv), bf16_hi_to_f32(hv)));
                const float2 lw = sub2(w, make_float2(bf16_lo_to_f32(hw), bf16_hi_to_f32(hw)));
                pa[8 + k] = pack_bf16(lv.x, lv.y);
                pb[8 + k] = pack_bf16(lw.x, lw.y);
            }
            if (ok) {
                tmem_st16(addr0, pa);
                tmem_st16(addr0 + 16, pb);
                tmem_wait_st();
                tc_fence_before();
            }
            __syncwarp();
            if (ok && lane == 0) mbar_arrive(&bar_p_full[buf][group]);
            // next item: kSlots groups further
            group += kSlots;
            while (group >= kGroups) {
                group -= kGroups;
                ++c;
                if (++buf == kBufs) {
                    buf = 0;
                    phase ^= 1u;
                }
            }
        }
        while (sg_next < nseg) {
            if (sg_next % kSlots == slot) run_epilogue(sg_next);
            ++sg_next;
        }
    }
    // ---------------------------------------------------------- teardown
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kLoadWarp) {
        if (s_abort) {
            // a wait gave up: give bulk copies and MMAs still in flight time to land
            // before the tensor memory and the shared buffers are released
            const long long t0 = clock64();
            while (clock64() - t0 < 4000000LL) {
            }
        }
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
    if (s_abort) return;  // a wait gave up: leave R and the selection as they are, err is set
    // tiles with no CTA (ntiles < grid) write nothing; CTAs without tiles still take a ticket
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(e.ticket, 1u) == gridDim.x - 1u) ? 1 : 0;
    __syncthreads();
    if (s_last) {
        __threadfence();
        epi_finalize<C>(e, red_d, red_i);
    }
}

// ---------------------------------------------------------- operand packing
namespace {

// byte offset of element (row, k) of a K-major, no-swizzle operand with KD
// columns: core matrices of 8 rows x 8 halves, K-adjacent cores 128 B apart.
__device__ __forceinline__ size_t core_off(int row, int k, int kd) {
    return ((size_t)((row >> 3) * (kd >> 3) + (k >> 3)) * 8 + (row & 7)) * 16 + (size_t)(k & 7) * 2;
}

__device__ __forceinline__ void split_f16(float v, __half& hi, __half& lo) {
    hi = __float2half_rn(v);
    lo = __float2half_rn(v - __half2float(hi));
}

// Value at K index k of the distance operand of a point with scaled (and
// log2(e)-folded) coordinates z[0..d) and a = |z|^2.  Rows (the tile's points):
// [z_hi | z_hi | z_lo | a_hi | a_lo | 1 | 1 | 0...]; columns (the block's
// points): [-2z_hi | -2z_lo | -2z_hi | 1 | 1 | a_hi | a_lo | 0...], so that the
// product of a row and a column sums the cross terms hi*hi + hi*lo + lo*hi and
// both squared norms.
__device__ __forceinline__ __half dist_operand(const double* z, double a, int d, int k, bool column) {
    __half hi, lo;
    if (k < 3 * d) {
        const int q = k % d, part = k / d;  // part 0, 1, 2
        split_f16((float)(column ? -2.0 * z[q] : z[q]), hi, lo);
        if (column) return part == 1 ? lo : hi;
        return part == 2 ? lo : hi;
    }
    const int r = k - 3 * d;
    if (r >= 4) return __float2half_rn(0.0f);
    split_f16((float)a, hi, lo);
    if (!column) return r == 0 ? hi : r == 1 ? lo : __float2half_rn(1.0f);
    return r < 2 ? __float2half_rn(1.0f) : (r == 2 ? hi : lo);
}

// Row operand tiles, for the rows of every block-aligned tile (zero rows past
// the end of a block).
__global__ void pack_rows_kernel(const float* __restrict__ Xs, int64_t n, int d, int D, int64_t b, int64_t tps,
                                 int kdp, float fold, uint8_t* __restrict__ XA) {
    const int64_t tile = blockIdx.x;
    const int64_t seg_lo = (tile / tps) * b;
    const int64_t seg_hi = min(seg_lo + b, n);
    const int64_t r0 = seg_lo + (tile % tps) * 128;
    uint8_t* dst = XA + (size_t)tile * 128 * kdp * 2;
    for (int t = threadIdx.x; t < 128 * kdp; t += blockDim.x) {
        const int row = t / kdp, k = t % kdp;
        const int64_t i = r0 + row;
        __half v = __float2half_rn(0.0f);
        if (i < seg_hi) {
            double z[AP_MAX_DIM], a = 0.0;
            for (int q = 0; q < d; ++q) {
                z[q] = (double)Xs[i * D + q] * fold;
                a += z[q] * z[q];
            }
            v = dist_operand(z, a, d, k, false);
        }
        *reinterpret_cast<__half*>(dst + core_off(row, k, kdp)) = v;
    }
}

// Column operand chunks: 128 columns per chunk, per block (zero past its end).
__global__ void pack_cols_kernel(const float* __restrict__ Xs, int64_t n, int d, int D, int64_t b, int cpb, int kdp,
                                 float fold, uint8_t* __restrict__ XB) {
    const int64_t chunk = blockIdx.x;  // block * cpb + q
    const int64_t blk = chunk / cpb;
    const int q = (int)(chunk % cpb);
    const int64_t lo_col = blk * b, hi_col = min(lo_col + b, n);
    uint8_t* dst = XB + (size_t)chunk * tc::kChunk * kdp * 2;
    for (int t = threadIdx.x; t < tc::kChunk * kdp; t += blockDim.x) {
        const int row = t / kdp, k = t % kdp;
        const int64_t j = lo_col + (int64_t)q * tc::kChunk + row;
        __half v = __float2half_rn(0.0f);
        if (j < hi_col) {
            double z[AP_MAX_DIM], a = 0.0;
            for (int s = 0; s < d; ++s) {
                z[s] = (double)Xs[j * D + s] * fold;
                a += z[s] * z[s];
            }
            v = dist_operand(z, a, d, k, true);
        }
        *reinterpret_cast<__half*>(dst + core_off(row, k, kdp)) = v;
    }
}

// Delta^T chunks of the current step: C rows (right-hand sides) x 128 columns
// (block-local points) as BF16 hi/lo, K-major core matrices of 8 rows x 8
// halves (16 K-cores per row group).
__global__ void pack_delta_kernel(const float* __restrict__ Delta, int64_t b, int C, int cpb, uint8_t* __restrict__ DT) {
    const int q = blockIdx.x;
    const size_t half_bytes = (size_t)C * tc::kChunk * 2;
    uint8_t* dst = DT + (size_t)q * 2 * half_bytes;
    for (int t = threadIdx.x; t < C * tc::kChunk; t += blockDim.x) {
        const int c = t / tc::kChunk, k = t % tc::kChunk;  // row c, K index k
        const int64_t li = (int64_t)q * tc::kChunk + k;
        const float v = li < b ? Delta[li * C + c] : 0.0f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        const size_t off =
            ((size_t)((c >> 3) * (tc::kChunk / 8) + (k >> 3)) * 8 + (c & 7)) * 16 + (size_t)(k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(dst + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(dst + half_bytes + off) = lo;
    }
}

template <int KERN, int C>
cudaError_t launch_tc_inst(const TcParams& p, int grid, cudaStream_t st) {
    const size_t xa = (size_t)tc::kRows * p.kdp * 2, xb = (size_t)tc::kChunk * p.kdp * 2;
    constexpr size_t dt = 2u * C * tc::kChunk * 2u;
    const size_t smem = 2 * xa + tc::kStages * (xb + dt) + 1024;
    auto fn = kmv_tc_kernel<KERN, C>;
    cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    fn<<<grid, tc::kThreads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

int tc_kd(int d) { return (3 * d + 4 + 15) / 16 * 16; }

int tc_chunks_per_block(int64_t b) { return (int)((b + tc::kChunk - 1) / tc::kChunk); }

size_t tc_rows_bytes(int64_t ntiles, int kd) { return (size_t)ntiles * 128 * kd * 2; }
size_t tc_cols_bytes(int64_t m, int cpb, int kd) { return (size_t)m * cpb * tc::kChunk * kd * 2; }
size_t tc_delta_bytes(int cpb, int C) { return (size_t)cpb * 2 * C * tc::kChunk * 2; }
size_t tc_share_bytes(int grid, int C) { return (size_t)grid * 2 * tc::kRows * C * sizeof(float); }

cudaError_t launch_tc_pack_inputs(int kernel, const float* Xs, int64_t n, int d, int D, int64_t b, int64_t m,
                                  int64_t tps, int cpb, int kd, uint8_t* XA, uint8_t* XB, cudaStream_t st) {
    const float fold = kernel == AP_RBF ? 1.0f : 1.4426950408889634f;
    pack_rows_kernel<<<(unsigned)(m * tps), 256, 0, st>>>(Xs, n, d, D, b, tps, kd, fold, XA);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    pack_cols_kernel<<<(unsigned)(m * cpb), 256, 0, st>>>(Xs, n, d, D, b, cpb, kd, fold, XB);
    return cudaGetLastError();
}

cudaError_t launch_tc_pack_delta(const float* Delta, int64_t b, int C, int cpb, uint8_t* DT, cudaStream_t st) {
    pack_delta_kernel<<<cpb, 256, 0, st>>>(Delta, b, C, cpb, DT);
    return cudaGetLastError();
}

cudaError_t launch_kmv_tc(int kernel, const TcParams& p, int C, int grid, cudaStream_t st) {
    if (p.kdp < 16 || p.kdp % 16 != 0 || p.kdp > kTcMaxKdp) return cudaErrorInvalidValue;
#define AP_TC_K(KK)                                                 \
    if (C == 16) return launch_tc_inst<KK, 16>(p, grid, st); \
    if (C == 32) return launch_tc_inst<KK, 32>(p, grid, st); \
    return cudaErrorInvalidValue;
    switch (kernel) {
        case AP_RBF: { AP_TC_K(AP_RBF) }
        case AP_MATERN32: { AP_TC_K(AP_MATERN32) }
        case AP_MATERN52: { AP_TC_K(AP_MATERN52) }
        default: return cudaErrorInvalidValue;
    }
#undef AP_TC_K
}

cudaError_t launch_kmv_tc_step(int kernel, const TcLaunch& l, int kd, int C, int grid, cudaStream_t st) {
    TcParams p;
    p.XA = l.XA;
    p.XB = l.XB;
    p.DT = l.DT;
    p.Delta = l.Delta;
    p.R = l.R;
    p.n = l.n;
    p.b = l.b;
    p.cpb = l.cpb;
    p.kdp = kd;
    p.s = l.s;
    p.noise = l.noise;
    p.sel = l.sel;
    p.err = l.err;
    p.wait_cycles = l.wait_cycles > 0 ? l.wait_cycles : tc::kWaitCycles;
    p.scr = l.scr;
    p.tick = l.tick;
    p.epi = l.epi;
    return launch_kmv_tc(kernel, p, C, grid, st);
}

}  // namespace ap
