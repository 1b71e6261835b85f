// Internal declarations shared by the CUDA translation units of libap.so.
// Nothing here is part of the public ABI (include/ap.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ap.h"

namespace ap {

// Bounds-checked build (compiled with -DAP_CHECKED into a separate library):
// AP_CHK(cond) guards an index before the access it protects.  A failing check
// records its source line in a device word of its translation unit (the first
// one wins) and yields false, so that the caller skips the access instead of
// faulting; ap_bounds_violations reads and clears the words of every unit.  In
// the product build AP_CHK(cond) is `true` and compiles away.
#ifdef AP_CHECKED
namespace {
__device__ unsigned int g_chk_line;  // one per translation unit
}
#define AP_CHK(cond) ((cond) ? true : (atomicCAS(&g_chk_line, 0u, (unsigned int)__LINE__), false))
// Host registry of the per-unit words (defined in ap_api.cu).
int chk_register(const char* unit, unsigned int (*read_and_clear)());
namespace {
unsigned int chk_read_and_clear() {
    unsigned int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_chk_line, sizeof v) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_chk_line, &zero, sizeof zero);
    return v;
}
const int g_chk_registered = chk_register(__BASE_FILE__, &chk_read_and_clear);
}  // namespace
#else
#define AP_CHK(cond) true
#endif

constexpr int kTile = 64;           // tile edge of the block-Cholesky cache
constexpr int kKmvThreads = 128;    // threads per CTA of the kernel-matrix products
constexpr int kKmvTN = 64;          // columns staged per shared-memory chunk
constexpr int kMaxSplit = 8;        // portable thread-block-cluster size

// flags of the kernel-matrix product epilogue
constexpr int kEpiBlockNorms = 1;   // per-block ||R_J||_F^2 partials + block selection
constexpr int kEpiColNorms = 2;     // per-column ||R_:,c||^2 partials

// Scale applied to x / l so that the FP32 kernels evaluate phi with one ex2:
//   RBF:  |x_s - x_s'|^2 = r^2 log2(e) / 2          -> phi = 2^(-|.|^2)
//   M32:  |x_s - x_s'|   = sqrt(3) r = u             -> phi = (1 + u) 2^(-u log2 e)
//   M52:  |x_s - x_s'|   = sqrt(5) r = u             -> phi = (1 + u + u^2/3) 2^(-u log2 e)
double kernel_input_scale(int kernel);

// Epilogue bookkeeping of one AP step (block norms, selection, column norms).
struct EpiParams {
    int flags;
    int advance;            // 1: a step finished (step_ctr += 1) before selecting
    int64_t seg;            // rows per AP block b (tiles never straddle a block)
    int64_t tiles_per_seg;  // CTA row tiles per block
    int64_t ntiles;         // row tiles in the grid (y dimension)
    int S;                  // CTAs per row tile (cluster size, x dimension)
    int m;                  // number of blocks
    double* part_norm;      // [ntiles * S]
    double* part_col;       // [ntiles * S * C]
    unsigned int* ticket;   // last-CTA counter, left at 0 after each launch
    double* norms_out;      // [m]   block norms after the step
    double* colnorm_out;    // [C]   column norms (when kEpiColNorms)
    int select;             // ap_select
    uint64_t seed;
    int64_t* step_ctr;      // steps completed (device)
    int* sel_out;           // block chosen for the next step (device)
    int* nan_flag;          // set to 1 when a norm is not finite
};

// out[i,:] = base[i,:] + sgn * s * sum_j phi(xa_i, xb_j) V[j - col0, :]
//            + sgn * noise * V[i - col0, :]   (if noise_diag and col0 <= i < col0 + ncols)
struct KmvParams {
    const float* Xa;       // na x D scaled rows
    int64_t na;
    const float* Xb;       // nb x D scaled columns
    int64_t nb;
    const float* V;        // ncols x C
    const float* base;     // na x C or nullptr (then base_const)
    float base_const;
    float* out;            // na x C (may alias base)
    float sgn;
    float s;
    float noise;
    int noise_diag;
    int64_t col0, ncols;   // column range when sel == nullptr
    const int* sel;        // device block index: col0 = sel*blk, ncols = min(blk, nb - col0)
    int64_t blk;
    const float* Xa_lo;    // compensated form only: low parts of the scaled inputs
    const float* Xb_lo;
    EpiParams epi;
};

// FP32 SIMT kernel-matrix product with the AP epilogue (one per kernel family TU).
cudaError_t launch_kmv_rbf(const KmvParams& p, int D, int C, cudaStream_t st);
cudaError_t launch_kmv_m32(const KmvParams& p, int D, int C, cudaStream_t st);
cudaError_t launch_kmv_m52(const KmvParams& p, int D, int C, cudaStream_t st);
cudaError_t launch_kmv(int kernel, const KmvParams& p, int D, int C, cudaStream_t st);
// Compensated (double-float FP32) form of the same product, for refinement.
cudaError_t launch_kmv_comp_rbf(const KmvParams& p, int D, int C, cudaStream_t st);
cudaError_t launch_kmv_comp_m32(const KmvParams& p, int D, int C, cudaStream_t st);
cudaError_t launch_kmv_comp_m52(const KmvParams& p, int D, int C, cudaStream_t st);
cudaError_t launch_kmv_comp(int kernel, const KmvParams& p, int D, int C, cudaStream_t st);
constexpr int kCompRows = 128;  // rows per CTA of the compensated product

// Rows per CTA for a (D, C) instance of the FP32 product.
int kmv_rows_per_cta(int D, int C);

// Norms of R alone (n x C) + selection: used before the first step and after refinement.
cudaError_t launch_norms_select(const float* R, int64_t n, int C, const EpiParams& e,
                                int64_t tile_rows, cudaStream_t st);

// ---- block-Cholesky cache (FP64 factorisation, FP32 inverse factor) --------
struct CacheParams {
    const float* X;        // n x d, original inputs
    int64_t n;
    int d;
    int kernel;
    double ell[AP_MAX_DIM];
    double s, noise;
    int64_t b;             // block size
    int nt;                // tiles per block edge = ceil(b / kTile)
};

// Factor blocks [blk0, blk0 + g) into the packed FP32 inverse factors Linv.
// A (g * (nt*64)^2 doubles) and Dinv (g * nt * 64^2 doubles) are work buffers.
// bad (g ints) gets 1 for a block whose factorisation met a non-positive pivot.
// Tensor-core panel solves and trailing updates with FP64 results (ozaki.cu): slice planes of
// oz_slice_bytes(nt) bytes and oz_expo_ints(nt) row exponents per block.
size_t oz_slice_bytes(int nt);
size_t oz_expo_ints(int nt);
cudaError_t launch_oz_update(double* A, int nt, int k, int g, uint8_t* S, int* E, int* err, cudaStream_t st,
                             int64_t* launches);
// The panel solve A_ik := A_ik L_kk^{-T} (i > k) the same way, L_kk^{-1} from Dinv.
cudaError_t launch_oz_trsm(double* A, const double* Dinv, int nt, int k, int g, uint8_t* S, int* E, int* err,
                           cudaStream_t st, int64_t* launches);
// Work buffers of the tensor-core panel solves and trailing updates; null = FP64 FMA.
struct OzWork {
    uint8_t* S;  // g * oz_slice_bytes(nt)
    int* E;      // g * oz_expo_ints(nt)
    int* err;    // wait-timeout flag
};
// FP64 phi of the cache build at count squared distances (device arrays).
cudaError_t launch_phi_fp64_eval(int kernel, const double* r2, int64_t count, double* out, cudaStream_t st);
cudaError_t cache_factor_group(const CacheParams& cp, int64_t blk0, int g, double* A, double* Dinv,
                               float* Linv, int* bad, const OzWork* oz, cudaStream_t st, int64_t* launches);

// ---- block solve: Delta = L^-T L^-1 R_I, W_I += Delta -----------------------
struct SolveParams {
    const float* Linv;     // packed inverse factors of all blocks
    int64_t n, b;
    int nt;
    int C;
    const float* R;        // n x C
    float* W;              // n x C
    float* Z;              // nt*64 x C work
    float* Delta;          // b x C (rows >= b_I are written as 0)
    const int* sel;
    const int64_t* step_ctr;
    int* trace;            // device trace or nullptr
    int64_t trace_cap;
    int tpc;               // tiles per CTA (block_solve_layout)
    int maxj;              // partial slots per output row of tiles
    float* spart;          // nt * maxj * 64 * max(C, 4) floats of partial sums
    unsigned* sticket;     // nt tickets, zero between launches
};
// Work split of the block solve for nt tiles per block edge on num_sms SMs.
void block_solve_layout(int nt, int num_sms, int* tpc, int* maxj);
cudaError_t launch_block_solve(const SolveParams& p, cudaStream_t st, int64_t* launches);

// ---- small helpers ----------------------------------------------------------
// Xs = fl(X * sc) with sc = sc_hi + sc_lo per dimension; Xs_lo (may be null)
// gets the remainder X * sc - Xs to FP32 precision.
cudaError_t launch_prep_inputs(const float* X, int64_t n, int d, int D, const float* sc_hi, const float* sc_lo,
                               float* Xs, float* Xs_lo, int* bad, cudaStream_t st);
cudaError_t launch_pad_copy(const float* src, int64_t n, int c, float* dst, int C, cudaStream_t st);
cudaError_t launch_unpad_copy(const float* src, int64_t n, int C, float* dst, int c, cudaStream_t st);

// ---- derivative quadratic forms (Eq. loss_grad_unbiased) ------------------
// Accumulates, over all pairs (i, j), G_ij = sum_c alpha_c U_ic V_jc times
//   out[k]     (k < D): G_ij psi(t_ij) (xs_ik - xs_jk)^2   (lengthscale terms)
//   out[D]:            G_ij phi(t_ij)                      (outputscale term)
//   out[D + 1]:        G_ii                                 (noise term)
// with the pre-scaled inputs xs of the FP32 product; the host turns these
// into dK/dtheta quadratic forms.
struct GradParams {
    const float* Xs;       // n x D scaled inputs
    int64_t n;
    const float* U;        // n x C
    const float* V;        // n x C
    float alpha[AP_MAX_RHS];
    int64_t ntiles;        // row tiles (grid.x)
    int S;                 // column splits (grid.y)
    double* part;          // [ntiles * S * (D + 2)]
    unsigned int* ticket;
    double* out;           // D + 2
};
cudaError_t launch_grad(int kernel, const GradParams& p, int D, int C, cudaStream_t st);
cudaError_t launch_grad_rbf(const GradParams& p, int D, int C, cudaStream_t st);
cudaError_t launch_grad_m32(const GradParams& p, int D, int C, cudaStream_t st);
cudaError_t launch_grad_m52(const GradParams& p, int D, int C, cudaStream_t st);
int grad_rows_per_cta(int D, int C);

// B = [y - mu, z_1..z_l]; Z == nullptr draws Rademacher z from SplitMix64(seed);
// Zout (may be nullptr) receives the z actually used.
cudaError_t launch_assemble_rhs(const float* y, float mu, const float* Z, int l, uint64_t seed, int64_t n,
                                float* B, float* Zout, cudaStream_t st);
// V = [W[:,0], B[:,1..c)] padded to C columns.
cudaError_t launch_assemble_v(const float* W, int C, const float* B, int c, int64_t n, float* V, cudaStream_t st);
// out = sum_i W[i*C] * (Y ? Y[i*cy] : 1) in FP64; part needs 256 doubles.
cudaError_t launch_dot0(const float* W, int C, const float* Y, int cy, int64_t n, double* part, unsigned* ticket,
                       double* out, cudaStream_t st);

// ---- tensor-core form of the residual update (kmv_tc.cu) -------------------
struct TcParams;
int tc_kd(int d);
int tc_chunks_per_block(int64_t b);
size_t tc_rows_bytes(int64_t ntiles, int kd);
size_t tc_cols_bytes(int64_t m, int cpb, int kd);
size_t tc_delta_bytes(int cpb, int C);
cudaError_t launch_tc_pack_inputs(int kernel, const float* Xs, int64_t n, int d, int D, int64_t b, int64_t m,
                                  int64_t tps, int cpb, int kd, uint8_t* XA, uint8_t* XB, cudaStream_t st);
cudaError_t launch_tc_pack_delta(const float* Delta, int64_t b, int C, int cpb, uint8_t* DT, cudaStream_t st);
struct TcLaunch {
    const uint8_t* XA;
    const uint8_t* XB;
    const uint8_t* DT;
    const float* Delta;
    float* R;
    int64_t n, b;
    int cpb;
    float s, noise;
    const int* sel;
    int* err;
    long long wait_cycles;  // bound of the kernel's waits (<= 0: the default, about 2 s)
    float* scr;  // grid x 2 x 128 x C floats (tc_share_bytes)
    int* tick;   // grid ints, zero
    EpiParams epi;
};
// Boundary slots of the tensor-core update for a grid of CTAs and C right-hand sides.
size_t tc_share_bytes(int grid, int C);
cudaError_t launch_kmv_tc_step(int kernel, const TcLaunch& l, int kd, int C, int grid, cudaStream_t st);

// Makes the context's device current for one call and restores the caller's.
class DeviceGuard {
   public:
    explicit DeviceGuard(int dev) {
        ok_ = cudaGetDevice(&prev_) == cudaSuccess;
        if (ok_ && prev_ != dev) ok_ = cudaSetDevice(dev) == cudaSuccess, switched_ = ok_;
        if (!ok_) cudaGetLastError();
    }
    ~DeviceGuard() {
        if (switched_) cudaSetDevice(prev_);
    }
    bool ok() const { return ok_; }

   private:
    int prev_ = 0;
    bool ok_ = false, switched_ = false;
};

// Read-only view of what the gradient kernel needs from a context.
struct GradView {
    int device;           // the context's device
    const float* Xs;
    int64_t n;
    int d, D, kernel;
    float s;
    const float* ell;
    cudaStream_t stream;  // the caller's stream of the context
};
void ctx_grad_view(const ap_ctx* ctx, GradView* v);
// Turn the raw D + 2 sums of the gradient kernel into the d + 2 quadratic forms.
void grad_finish(const GradView& v, const double* raw, double* out_host);

}  // namespace ap
