// Host orchestration and the exported C ABI (include/ap.h).
//
// Alg. 1 runs as: [block solve (2 kernels) -> fused residual update with the
// norm/selection epilogue (1 kernel)] per inner step, the block index living
// in device memory.  A whole epoch of m steps is captured once into a CUDA
// graph and replayed; the host reads only the c column norms at the end of an
// epoch to apply the stopping rule of Sec. 5.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ap_internal.cuh"

using namespace ap;

namespace {
// Named host-side range of one phase (cache, solve, epoch, refinement,
// prediction, gradient) for profilers and timeline tools; free when no tool
// is attached.
class PhaseRange {
   public:
    explicit PhaseRange(const char* name) { nvtxRangePushA(name); }
    ~PhaseRange() { nvtxRangePop(); }
    PhaseRange(const PhaseRange&) = delete;
    PhaseRange& operator=(const PhaseRange&) = delete;
};
}  // namespace

struct ap_ctx {
    int device = 0;  // current device at ap_create; every call runs with it current
    int64_t n = 0;
    int d = 0, D = 0;
    const float* X = nullptr;
    int kernel = 0;
    float ell[AP_MAX_DIM] = {};
    float s = 1.f, noise = 0.f, mean = 0.f;
    ap_opts o = {};
    cudaStream_t ust = nullptr;  // caller's stream
    cudaStream_t st = nullptr;   // context stream (work is ordered after ust on entry)
    cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_sync = nullptr;
    int64_t b = 0, m = 0;
    int nt = 0;
    int64_t ntri = 0;
    float* Xs = nullptr;
    float* Xs_lo = nullptr;  // remainders of the scaled inputs (compensated recompute)
    float* Linv = nullptr;
    size_t bytes = 0;
    std::unordered_map<void*, size_t> sizes;
    double t_cache = 0.0;
    // per-solve buffers (stride Cp)
    int Cp = 0;
    float *R = nullptr, *W = nullptr, *Bp = nullptr, *Z = nullptr, *Delta = nullptr, *Tmp = nullptr;
    float* W_ckpt = nullptr;  // low-precision forms: W at the last refinement that lowered the true residual
    double *part_norm = nullptr, *part_col = nullptr;
    int64_t part_alloc = 0;
    // block-solve work split and partial sums
    float* spart = nullptr;
    unsigned* sticket = nullptr;
    int sol_tpc = 1, sol_maxj = 1;
    // always-present device scalars
    double *norms = nullptr, *colnorm = nullptr, *gout = nullptr, *gpart = nullptr;
    int64_t gpart_alloc = 0;
    unsigned* ticket = nullptr;
    int* sel = nullptr;
    int64_t* step = nullptr;
    int* nan_flag = nullptr;
    int* bad = nullptr;
    int* trace = nullptr;
    int64_t trace_alloc = 0;
    float* Xt = nullptr;  // scaled test inputs
    int64_t Xt_alloc = 0;
    cudaGraphExec_t graph = nullptr;
    bool graph_broken = false;
    // per-kernel timing (opts.profile): events around each block solve / update of an epoch
    std::vector<cudaEvent_t> ev_bs, ev_up;
    double t_update = 0.0, t_bsolve = 0.0;
    int64_t n_update = 0;
    cudaEvent_t ev_r0 = nullptr, ev_r1 = nullptr;
    // tensor-core form (AP_BF16_REFINE)
    bool tc = false;
    bool tc_steps = false;  // the current solve's steps use the tensor-core update (false after escalation)
    bool graph_tc = false;  // form of the steps in the captured epoch graph
    int kd = 16, cpb = 0, num_sms = 152;
    int64_t tps128 = 0;
    uint8_t *XA = nullptr, *XB = nullptr, *DT = nullptr;
    float* tc_scr = nullptr;  // boundary slots of tiles shared by two CTAs
    int* tc_tick = nullptr;
    int* tc_err = nullptr;
    int64_t launches = 0;
    int r_tracked_c = 0;  // c of the solve whose residual R holds (0: none)
    int divergences = 0;  // low-precision runs rolled back to a checkpoint (this solve)
    bool comp_auto = false;  // AP_RESID_AUTO switched this solve's recomputes to the compensated form
    bool comp_used = false;  // the last recompute was compensated
    cudaError_t last_cuda = cudaSuccess;
};

namespace {

#define AP_CK(expr)                                       \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) {                          \
            ctx->last_cuda = _e;                          \
            cudaGetLastError();                           \
            return AP_ERR_CUDA;                           \
        }                                                 \
    } while (0)

#define AP_DEVICE_GUARD(ctx)               \
    DeviceGuard _dg((ctx)->device);        \
    if (!_dg.ok()) return AP_ERR_CUDA

#define AP_TRY(expr)                       \
    do {                                   \
        ap_status _s = (expr);             \
        if (_s != AP_OK) return _s;        \
    } while (0)

int pad_c(int c) { return c <= 1 ? 1 : (c <= 4 ? 4 : (c <= 16 ? 16 : 32)); }
int pad_d(int d) {
    const int opts[] = {4, 8, 12, 16, 24, 32};
    for (int v : opts)
        if (d <= v) return v;
    return 32;
}

ap_status dalloc(ap_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (ctx->o.hbm_budget && ctx->bytes + bytes > ctx->o.hbm_budget) return AP_ERR_NOMEM;
    // stream-ordered allocation on the context stream: no device-wide
    // synchronisation, so concurrent contexts (serving) keep running
    if (cudaMallocAsync(p, bytes, ctx->st) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return AP_ERR_NOMEM;
    }
    ctx->bytes += bytes;
    ctx->sizes[*p] = bytes;
    return AP_OK;
}

template <class T>
ap_status dalloc_t(ap_ctx* ctx, T** p, size_t count) {
    return dalloc(ctx, reinterpret_cast<void**>(p), count * sizeof(T));
}

template <class T>
void dfree(ap_ctx* ctx, T*& p) {
    if (!p) return;
    auto it = ctx->sizes.find((void*)p);
    if (it != ctx->sizes.end()) {
        ctx->bytes -= it->second;
        ctx->sizes.erase(it);
    }
    cudaFreeAsync((void*)p, ctx->st);
    p = nullptr;
}

void drop_graph(ap_ctx* ctx) {
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
}

// Order the context stream after the caller's stream.
ap_status enter(ap_ctx* ctx) {
    AP_CK(cudaEventRecord(ctx->ev_sync, ctx->ust));
    AP_CK(cudaStreamWaitEvent(ctx->st, ctx->ev_sync, 0));
    return AP_OK;
}

// Finish the call: the caller's stream is ordered after our work and we wait.
ap_status leave(ap_ctx* ctx) {
    AP_CK(cudaEventRecord(ctx->ev_sync, ctx->st));
    AP_CK(cudaStreamWaitEvent(ctx->ust, ctx->ev_sync, 0));
    AP_CK(cudaStreamSynchronize(ctx->st));
    return AP_OK;
}

int choose_split(int64_t ntiles, int64_t ncols) {
    int S = 1;
    while (S < kMaxSplit && ntiles * S < 4 * 152 && ncols / (2 * S) >= kKmvTN) S *= 2;
    return S;
}

struct Shape {
    int64_t rows, tps, ntiles;
    int S;
};

// Row tiling of an AP-step product over the n training rows.
Shape step_shape(const ap_ctx* ctx, int Cp, int64_t ncols) {
    Shape sh;
    sh.rows = kmv_rows_per_cta(ctx->D, Cp);
    sh.tps = (ctx->b + sh.rows - 1) / sh.rows;
    sh.ntiles = ctx->m * sh.tps;
    sh.S = choose_split(sh.ntiles, ncols);
    return sh;
}

// Row tiling of the compensated recompute (one row per thread).
Shape comp_shape(const ap_ctx* ctx, int64_t ncols) {
    Shape sh;
    sh.rows = kCompRows;
    sh.tps = (ctx->b + sh.rows - 1) / sh.rows;
    sh.ntiles = ctx->m * sh.tps;
    sh.S = choose_split(sh.ntiles, ncols);
    return sh;
}

constexpr int64_t kNormRows = 512;

Shape norm_shape(const ap_ctx* ctx) {
    Shape sh;
    sh.rows = kNormRows;
    sh.tps = (ctx->b + kNormRows - 1) / kNormRows;
    sh.ntiles = ctx->m * sh.tps;
    sh.S = 1;
    return sh;
}

EpiParams make_epi(ap_ctx* ctx, int flags, int advance, const Shape& sh) {
    EpiParams e = {};
    e.flags = flags;
    e.advance = advance;
    e.seg = ctx->b;
    e.tiles_per_seg = sh.tps;
    e.ntiles = sh.ntiles;
    e.S = sh.S;
    e.m = (int)ctx->m;
    e.part_norm = ctx->part_norm;
    e.part_col = ctx->part_col;
    e.ticket = ctx->ticket;
    e.norms_out = ctx->norms;
    e.colnorm_out = ctx->colnorm;
    e.select = ctx->o.select;
    e.seed = ctx->o.seed;
    e.step_ctr = ctx->step;
    e.sel_out = ctx->sel;
    e.nan_flag = ctx->nan_flag;
    return e;
}

ap_status prep_inputs(ap_ctx* ctx, const float* X, int64_t n, float* out, float* out_lo) {
    float sh[AP_MAX_DIM] = {}, sl[AP_MAX_DIM] = {};
    const double ks = kernel_input_scale(ctx->kernel);
    for (int k = 0; k < ctx->d; ++k) {
        const double sc = ks / (double)ctx->ell[k];
        sh[k] = (float)sc;
        sl[k] = (float)(sc - (double)sh[k]);
    }
    AP_CK(launch_prep_inputs(X, n, ctx->d, ctx->D, sh, sl, out, out_lo, ctx->nan_flag, ctx->st));
    ++ctx->launches;
    return AP_OK;
}

bool use_compensated(const ap_ctx* ctx) {
    if (ctx->o.residual_mode == AP_RESID_COMPENSATED) return true;
    if (ctx->o.residual_mode == AP_RESID_FP32) return false;
    return ctx->o.tol <= 1e-5 || ctx->comp_auto;
}

ap_status build_cache(ap_ctx* ctx) {
    PhaseRange range("ap: Cholesky cache (prep, K_II, FP64 factor, inverse)");
    drop_graph(ctx);
    AP_CK(cudaMemsetAsync(ctx->nan_flag, 0, sizeof(int), ctx->st));
    AP_TRY(prep_inputs(ctx, ctx->X, ctx->n, ctx->Xs, ctx->Xs_lo));
    if (ctx->tc) {
        AP_CK(launch_tc_pack_inputs(ctx->kernel, ctx->Xs, ctx->n, ctx->d, ctx->D, ctx->b, ctx->m, ctx->tps128, ctx->cpb, ctx->kd,
                                    ctx->XA, ctx->XB, ctx->st));
        ctx->launches += 2;
    }
    const int64_t tile_elems = (int64_t)kTile * kTile;
    if (!ctx->Linv) AP_TRY(dalloc_t(ctx, &ctx->Linv, (size_t)(ctx->m * ctx->ntri * tile_elems)));
    const int64_t edge = (int64_t)ctx->nt * kTile;
    const bool emulate = ctx->o.cache_gemm == AP_CACHE_TC_EXACT;
    const size_t per_block = (size_t)(edge * edge + ctx->nt * tile_elems) * sizeof(double) +
                             (emulate ? oz_slice_bytes(ctx->nt) + oz_expo_ints(ctx->nt) * sizeof(int) : 0);
    // FP64 workspace of at most 16 GiB (or what the HBM budget leaves): as many
    // blocks per group as fit, the groups of equal size (every group pays the
    // same chain of dependent launches, however few blocks it holds)
    size_t cap = (size_t)16 << 30;
    if (ctx->o.hbm_budget) {
        const size_t left = ctx->o.hbm_budget > ctx->bytes ? ctx->o.hbm_budget - ctx->bytes : 0;
        cap = std::min(cap, left);
    }
    int64_t g = (int64_t)(cap / per_block);
    if (g < 1) return AP_ERR_NOMEM;
    g = std::min<int64_t>(g, ctx->m);
    g = std::min<int64_t>(g, 65535);
    const int64_t ngroups = (ctx->m + g - 1) / g;
    g = (ctx->m + ngroups - 1) / ngroups;
    double* A = nullptr;
    double* Dinv = nullptr;
    AP_TRY(dalloc_t(ctx, &A, (size_t)(g * edge * edge)));
    ap_status s = dalloc_t(ctx, &Dinv, (size_t)(g * ctx->nt * tile_elems));
    if (s != AP_OK) {
        dfree(ctx, A);
        return s;
    }
    uint8_t* ozS = nullptr;
    int* ozE = nullptr;
    if (emulate) {
        s = dalloc_t(ctx, &ozS, (size_t)g * oz_slice_bytes(ctx->nt));
        if (s == AP_OK) s = dalloc_t(ctx, &ozE, (size_t)g * oz_expo_ints(ctx->nt));
        if (s != AP_OK) {
            dfree(ctx, ozS);
            dfree(ctx, A);
            dfree(ctx, Dinv);
            return s;
        }
    }
    const OzWork oz = {ozS, ozE, ctx->tc_err};
    AP_CK(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->st));
    AP_CK(cudaMemsetAsync(ctx->bad, 0, sizeof(int) * ctx->m, ctx->st));
    CacheParams cp = {};
    cp.X = ctx->X;
    cp.n = ctx->n;
    cp.d = ctx->d;
    cp.kernel = ctx->kernel;
    for (int k = 0; k < ctx->d; ++k) cp.ell[k] = (double)ctx->ell[k];
    cp.s = ctx->s;
    cp.noise = ctx->noise;
    cp.b = ctx->b;
    cp.nt = ctx->nt;
    AP_CK(cudaEventRecord(ctx->ev_a, ctx->st));
    cudaError_t err = cudaSuccess;
    for (int64_t blk0 = 0; blk0 < ctx->m && err == cudaSuccess; blk0 += g) {
        const int gg = (int)std::min<int64_t>(g, ctx->m - blk0);
        err = cache_factor_group(cp, blk0, gg, A, Dinv, ctx->Linv, ctx->bad + blk0, emulate ? &oz : nullptr, ctx->st,
                                 &ctx->launches);
    }
    AP_CK(err);
    AP_CK(cudaEventRecord(ctx->ev_b, ctx->st));
    AP_CK(cudaStreamSynchronize(ctx->st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b);
    ctx->t_cache = ms * 1e-3;
    dfree(ctx, A);
    dfree(ctx, Dinv);
    dfree(ctx, ozS);
    dfree(ctx, ozE);
    int tmo = 0, nanx = 0;
    AP_CK(cudaMemcpy(&tmo, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    AP_CK(cudaMemcpy(&nanx, ctx->nan_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (nanx) return AP_ERR_NAN;  // a NaN or Inf training input
    if (tmo) return AP_ERR_TIMEOUT;
    std::vector<int> bad((size_t)ctx->m);
    AP_CK(cudaMemcpy(bad.data(), ctx->bad, sizeof(int) * ctx->m, cudaMemcpyDeviceToHost));
    for (int64_t J = 0; J < ctx->m; ++J)
        if (bad[(size_t)J]) return AP_ERR_NOT_SPD;
    return AP_OK;
}

int first_bad_block(ap_ctx* ctx) {
    std::vector<int> bad((size_t)ctx->m);
    if (cudaMemcpy(bad.data(), ctx->bad, sizeof(int) * ctx->m, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    for (int64_t J = 0; J < ctx->m; ++J)
        if (bad[(size_t)J]) return (int)J;
    return -1;
}

ap_status ensure_solve(ap_ctx* ctx, int Cp) {
    if (ctx->Cp != Cp) {
        drop_graph(ctx);
        dfree(ctx, ctx->R);
        dfree(ctx, ctx->W);
        dfree(ctx, ctx->Bp);
        dfree(ctx, ctx->Z);
        dfree(ctx, ctx->Delta);
        dfree(ctx, ctx->Tmp);
        dfree(ctx, ctx->W_ckpt);
        dfree(ctx, ctx->part_col);
        dfree(ctx, ctx->spart);
        dfree(ctx, ctx->sticket);
        ctx->Cp = 0;
        ctx->r_tracked_c = 0;
        const size_t nc = (size_t)(ctx->n * Cp);
        AP_TRY(dalloc_t(ctx, &ctx->R, nc));
        AP_TRY(dalloc_t(ctx, &ctx->W, nc));
        AP_TRY(dalloc_t(ctx, &ctx->Bp, nc));
        AP_TRY(dalloc_t(ctx, &ctx->Tmp, nc));
        if (ctx->tc) AP_TRY(dalloc_t(ctx, &ctx->W_ckpt, nc));
        AP_TRY(dalloc_t(ctx, &ctx->Z, (size_t)ctx->nt * kTile * Cp));
        AP_TRY(dalloc_t(ctx, &ctx->Delta, (size_t)ctx->b * Cp));
        block_solve_layout(ctx->nt, ctx->num_sms, &ctx->sol_tpc, &ctx->sol_maxj);
        AP_TRY(dalloc_t(ctx, &ctx->spart, (size_t)ctx->nt * ctx->sol_maxj * kTile * std::max(Cp, 4)));
        AP_TRY(dalloc_t(ctx, &ctx->sticket, (size_t)ctx->nt));
        AP_CK(cudaMemsetAsync(ctx->sticket, 0, sizeof(unsigned) * ctx->nt, ctx->st));
        const Shape a = step_shape(ctx, Cp, ctx->b), b = step_shape(ctx, Cp, ctx->n), c = norm_shape(ctx);
        const Shape d = comp_shape(ctx, ctx->n);
        int64_t need = std::max(std::max(a.ntiles * a.S, b.ntiles * b.S), std::max(c.ntiles, d.ntiles * d.S));
        need = std::max(need, ctx->m * ctx->tps128);
        if (ctx->tc) {
            dfree(ctx, ctx->DT);
            AP_TRY(dalloc_t(ctx, &ctx->DT, tc_delta_bytes(ctx->cpb, Cp)));
        }
        dfree(ctx, ctx->part_norm);
        AP_TRY(dalloc_t(ctx, &ctx->part_norm, (size_t)need));
        AP_TRY(dalloc_t(ctx, &ctx->part_col, (size_t)need * Cp));
        ctx->part_alloc = need;
        ctx->Cp = Cp;
    }
    return AP_OK;
}

// One AP inner step: block solve, then the fused residual update whose
// epilogue selects the next block (and sums the column norms if colnorms).
ap_status launch_step(ap_ctx* ctx, bool colnorms, int64_t j) {
    const int Cp = ctx->Cp;
    const bool prof = ctx->o.profile && (size_t)(2 * j + 1) < ctx->ev_up.size();
    // timing events: external event nodes while an epoch is being captured
    // into a graph, plain records when the steps are launched directly
    unsigned rec_flags = cudaEventRecordDefault;
    if (prof) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        AP_CK(cudaStreamIsCapturing(ctx->st, &cs));
        if (cs == cudaStreamCaptureStatusActive) rec_flags = cudaEventRecordExternal;
    }
    if (prof) AP_CK(cudaEventRecordWithFlags(ctx->ev_bs[2 * j], ctx->st, rec_flags));
    SolveParams sp = {};
    sp.Linv = ctx->Linv;
    sp.n = ctx->n;
    sp.b = ctx->b;
    sp.nt = ctx->nt;
    sp.C = Cp;
    sp.R = ctx->R;
    sp.W = ctx->W;
    sp.Z = ctx->Z;
    sp.Delta = ctx->Delta;
    sp.sel = ctx->sel;
    sp.step_ctr = ctx->step;
    sp.trace = ctx->trace;
    sp.trace_cap = ctx->trace_alloc;
    sp.tpc = ctx->sol_tpc;
    sp.maxj = ctx->sol_maxj;
    sp.spart = ctx->spart;
    sp.sticket = ctx->sticket;
    AP_CK(launch_block_solve(sp, ctx->st, &ctx->launches));
    if (ctx->tc_steps) {
        AP_CK(launch_tc_pack_delta(ctx->Delta, ctx->b, Cp, ctx->cpb, ctx->DT, ctx->st));
        ++ctx->launches;
    }
    if (prof) {
        AP_CK(cudaEventRecordWithFlags(ctx->ev_bs[2 * j + 1], ctx->st, rec_flags));
        AP_CK(cudaEventRecordWithFlags(ctx->ev_up[2 * j], ctx->st, rec_flags));
    }
    if (ctx->tc_steps) {
        Shape sh;
        sh.rows = 128;
        sh.tps = ctx->tps128;
        sh.ntiles = ctx->m * ctx->tps128;
        sh.S = 1;
        TcLaunch tl = {};
        tl.XA = ctx->XA;
        tl.XB = ctx->XB;
        tl.DT = ctx->DT;
        tl.Delta = ctx->Delta;
        tl.R = ctx->R;
        tl.n = ctx->n;
        tl.b = ctx->b;
        tl.cpb = ctx->cpb;
        tl.s = ctx->s;
        tl.noise = ctx->noise;
        tl.sel = ctx->sel;
        tl.err = ctx->tc_err;
        tl.wait_cycles = ctx->o.wait_limit_cycles;
        tl.scr = ctx->tc_scr;
        tl.tick = ctx->tc_tick;
        tl.epi = make_epi(ctx, kEpiBlockNorms | (colnorms ? kEpiColNorms : 0), 1, sh);
        const int grid = (int)std::min<int64_t>(ctx->num_sms, sh.ntiles);
        AP_CK(launch_kmv_tc_step(ctx->kernel, tl, ctx->kd, Cp, grid, ctx->st));
        ++ctx->launches;
        if (prof) AP_CK(cudaEventRecordWithFlags(ctx->ev_up[2 * j + 1], ctx->st, rec_flags));
        return AP_OK;
    }
    const Shape sh = step_shape(ctx, Cp, ctx->b);
    KmvParams kp = {};
    kp.Xa = ctx->Xs;
    kp.na = ctx->n;
    kp.Xb = ctx->Xs;
    kp.nb = ctx->n;
    kp.V = ctx->Delta;
    kp.base = ctx->R;
    kp.out = ctx->R;
    kp.sgn = -1.f;
    kp.s = ctx->s;
    kp.noise = ctx->noise;
    kp.noise_diag = 1;
    kp.sel = ctx->sel;
    kp.blk = ctx->b;
    kp.epi = make_epi(ctx, kEpiBlockNorms | (colnorms ? kEpiColNorms : 0), 1, sh);
    AP_CK(launch_kmv(ctx->kernel, kp, ctx->D, Cp, ctx->st));
    ++ctx->launches;
    if (prof) AP_CK(cudaEventRecordWithFlags(ctx->ev_up[2 * j + 1], ctx->st, rec_flags));
    return AP_OK;
}

// Sum the per-step event pairs of the epoch that just finished (stream synced).
void collect_profile(ap_ctx* ctx, int64_t steps) {
    if (!ctx->o.profile) return;
    for (int64_t j = 0; j < steps && (size_t)(2 * j + 1) < ctx->ev_up.size(); ++j) {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, ctx->ev_up[2 * j], ctx->ev_up[2 * j + 1]) == cudaSuccess) {
            ctx->t_update += a * 1e-3;
            ++ctx->n_update;
        }
        if (cudaEventElapsedTime(&b, ctx->ev_bs[2 * j], ctx->ev_bs[2 * j + 1]) == cudaSuccess)
            ctx->t_bsolve += b * 1e-3;
    }
    cudaGetLastError();
}

// out = base - K_hat V over all n columns (the FP32 residual recompute).
ap_status launch_full_residual(ap_ctx* ctx, const float* base, const float* V, float* out, int flags) {
    PhaseRange range("ap: residual recompute R = B - K_hat W");
    const bool comp = use_compensated(ctx);
    ctx->comp_used = comp;
    const Shape sh = comp ? comp_shape(ctx, ctx->n) : step_shape(ctx, ctx->Cp, ctx->n);
    KmvParams kp = {};
    kp.Xa = ctx->Xs;
    kp.na = ctx->n;
    kp.Xb = ctx->Xs;
    kp.nb = ctx->n;
    kp.V = V;
    kp.base = base;
    kp.out = out;
    kp.sgn = -1.f;
    kp.s = ctx->s;
    kp.noise = ctx->noise;
    kp.noise_diag = 1;
    kp.col0 = 0;
    kp.ncols = ctx->n;
    kp.Xa_lo = ctx->Xs_lo;
    kp.Xb_lo = ctx->Xs_lo;
    kp.epi = make_epi(ctx, flags, 0, sh);
    if (comp) AP_CK(launch_kmv_comp(ctx->kernel, kp, ctx->D, ctx->Cp, ctx->st));
    else AP_CK(launch_kmv(ctx->kernel, kp, ctx->D, ctx->Cp, ctx->st));
    ++ctx->launches;
    return AP_OK;
}

ap_status launch_norms(ap_ctx* ctx, const float* R, int flags) {
    const Shape sh = norm_shape(ctx);
    EpiParams e = make_epi(ctx, flags, 0, sh);
    AP_CK(launch_norms_select(R, ctx->n, ctx->Cp, e, sh.rows, ctx->st));
    ++ctx->launches;
    return AP_OK;
}

ap_status run_epoch(ap_ctx* ctx, int64_t steps) {
    const bool full = steps == ctx->m;
    if (full && !ctx->graph_broken) {
        if (!ctx->graph) {
            cudaGraph_t g = nullptr;
            const int64_t l0 = ctx->launches;
            if (cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                ap_status s = AP_OK;
                for (int64_t j = 0; j < steps && s == AP_OK; ++j) s = launch_step(ctx, j == steps - 1, j);
                cudaError_t e = cudaStreamEndCapture(ctx->st, &g);
                if (s == AP_OK && e == cudaSuccess && g) {
                    if (cudaGraphInstantiate(&ctx->graph, g, 0) != cudaSuccess) ctx->graph = nullptr;
                    ctx->graph_tc = ctx->tc_steps;
                }
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();
            ctx->launches = l0;
            if (!ctx->graph) ctx->graph_broken = true;
        }
        if (ctx->graph) {
            AP_CK(cudaGraphLaunch(ctx->graph, ctx->st));
            ctx->launches += (ctx->tc_steps ? 4 : 3) * steps;
            return AP_OK;
        }
    }
    for (int64_t j = 0; j < steps; ++j) AP_TRY(launch_step(ctx, j == steps - 1, j));
    return AP_OK;
}

bool stop_met(int rule, double tol, int c, const double* rel, double fro_r, double fro_b) {
    if (rule == AP_STOP_FRO) return fro_r <= tol * fro_b;
    if (rule == AP_STOP_Y_REL) return rel[0] <= tol;
    if (rule == AP_STOP_MAX_REL) {
        for (int k = 0; k < c; ++k)
            if (!(rel[k] <= tol)) return false;
        return true;
    }
    double mean = 0.0;
    for (int k = 0; k < c; ++k) mean += rel[k];
    return mean / c < tol;
}

// The quantity the stopping rule compares with tol, from per-column relative
// residuals (FRO weights each column by ||b_c||^2).
double rule_measure(int rule, int c, const double* rel, const double* bn) {
    if (rule == AP_STOP_Y_REL) return rel[0];
    double acc = 0.0, w = 0.0;
    for (int k = 0; k < c; ++k) {
        if (rule == AP_STOP_MAX_REL) acc = std::max(acc, rel[k]);
        else if (rule == AP_STOP_FRO) acc += rel[k] * rel[k] * bn[k], w += bn[k];
        else acc += rel[k];
    }
    if (rule == AP_STOP_FRO) return w > 0.0 ? sqrt(acc / w) : sqrt(acc);
    return rule == AP_STOP_MAX_REL ? acc : acc / c;
}

ap_status check_hyper(const ap_hyper* h, int d) {
    if (!h || h->d != d || !h->lengthscale) return AP_ERR_INVALID_ARG;
    if (h->kernel != AP_RBF && h->kernel != AP_MATERN32 && h->kernel != AP_MATERN52) return AP_ERR_INVALID_ARG;
    for (int k = 0; k < d; ++k)
        if (!(h->lengthscale[k] > 0.f) || !isfinite(h->lengthscale[k])) return AP_ERR_INVALID_ARG;
    if (!(h->outputscale > 0.f) || !isfinite(h->outputscale)) return AP_ERR_INVALID_ARG;
    if (!(h->noise >= 0.f) || !isfinite(h->noise) || !isfinite(h->mean)) return AP_ERR_INVALID_ARG;
    return AP_OK;
}

void copy_hyper(ap_ctx* ctx, const ap_hyper* h) {
    ctx->kernel = h->kernel;
    for (int k = 0; k < ctx->d; ++k) ctx->ell[k] = h->lengthscale[k];
    ctx->s = h->outputscale;
    ctx->noise = h->noise;
    ctx->mean = h->mean;
}

void free_all(ap_ctx* ctx) {
    drop_graph(ctx);
    std::vector<void*> ptrs;
    for (auto& kv : ctx->sizes) ptrs.push_back(kv.first);
    for (void* p : ptrs) cudaFreeAsync(p, ctx->st);
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    ctx->sizes.clear();
    ctx->bytes = 0;
    if (ctx->ev_a) cudaEventDestroy(ctx->ev_a);
    if (ctx->ev_b) cudaEventDestroy(ctx->ev_b);
    if (ctx->ev_sync) cudaEventDestroy(ctx->ev_sync);
    if (ctx->ev_r0) cudaEventDestroy(ctx->ev_r0);
    if (ctx->ev_r1) cudaEventDestroy(ctx->ev_r1);
    for (cudaEvent_t e : ctx->ev_bs) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->ev_up) cudaEventDestroy(e);
    ctx->ev_bs.clear();
    ctx->ev_up.clear();
    if (ctx->st) cudaStreamDestroy(ctx->st);
    cudaGetLastError();
}

int solve_width(const ap_ctx* ctx, int c) { return ctx->tc ? std::max(16, pad_c(c)) : pad_c(c); }

ap_status solve_impl(ap_ctx* ctx, const float* B_dev, int c, const float* W0_dev, float* W_dev, ap_info* info) {
    PhaseRange range("ap: solve (Alg. 1)");
    const int Cp = solve_width(ctx, c);
    AP_TRY(ensure_solve(ctx, Cp));
    const int64_t want_trace = ctx->o.block_trace ? ctx->o.trace_cap : 0;
    if (want_trace > ctx->trace_alloc) {
        drop_graph(ctx);
        dfree(ctx, ctx->trace);
        ctx->trace_alloc = 0;
        AP_TRY(dalloc_t(ctx, &ctx->trace, (size_t)want_trace));
        ctx->trace_alloc = want_trace;
    }
    const int64_t l0 = ctx->launches;
    ctx->r_tracked_c = 0;
    ctx->tc_steps = ctx->tc;
    ctx->comp_auto = false;
    ctx->divergences = 0;
    if (ctx->graph && ctx->graph_tc != ctx->tc_steps) drop_graph(ctx);
    int fp32_epochs = 0;
    AP_TRY(enter(ctx));
    AP_CK(launch_pad_copy(B_dev, ctx->n, c, ctx->Bp, Cp, ctx->st));
    ++ctx->launches;
    AP_CK(cudaMemsetAsync(ctx->step, 0, sizeof(int64_t), ctx->st));
    AP_CK(cudaMemsetAsync(ctx->nan_flag, 0, sizeof(int), ctx->st));
    AP_CK(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->st));
    // arrival tickets start at zero (a launch that gave up on a wait leaves them partial)
    AP_CK(cudaMemsetAsync(ctx->ticket, 0, 4 * sizeof(unsigned), ctx->st));
    if (ctx->tc_tick) AP_CK(cudaMemsetAsync(ctx->tc_tick, 0, sizeof(int) * ctx->num_sms, ctx->st));
    // ||b_c|| for the relative residuals
    AP_TRY(launch_norms(ctx, ctx->Bp, kEpiColNorms));
    double bn[AP_MAX_RHS] = {}, rn[AP_MAX_RHS] = {};
    AP_CK(cudaMemcpyAsync(bn, ctx->colnorm, sizeof(double) * Cp, cudaMemcpyDeviceToHost, ctx->st));
    if (W0_dev) {
        AP_CK(launch_pad_copy(W0_dev, ctx->n, c, ctx->W, Cp, ctx->st));
        ++ctx->launches;
        AP_TRY(launch_full_residual(ctx, ctx->Bp, ctx->W, ctx->R, 0));
    } else {
        AP_CK(cudaMemsetAsync(ctx->W, 0, sizeof(float) * ctx->n * Cp, ctx->st));
        AP_CK(cudaMemcpyAsync(ctx->R, ctx->Bp, sizeof(float) * ctx->n * Cp, cudaMemcpyDeviceToDevice, ctx->st));
    }
    AP_TRY(launch_norms(ctx, ctx->R, kEpiBlockNorms | kEpiColNorms));
    AP_CK(cudaMemcpyAsync(rn, ctx->colnorm, sizeof(double) * Cp, cudaMemcpyDeviceToHost, ctx->st));
    if (ctx->tc)
        AP_CK(cudaMemcpyAsync(ctx->W_ckpt, ctx->W, sizeof(float) * ctx->n * Cp, cudaMemcpyDeviceToDevice, ctx->st));
    AP_CK(cudaStreamSynchronize(ctx->st));

    double rel[AP_MAX_RHS] = {}, rel_true[AP_MAX_RHS] = {};
    bool have_true = false;
    int true_epoch = -1;  // epoch at which rel_true was last recomputed
    int epoch = 0, refinements = 0;
    int64_t steps = 0;
    double t_refine = 0.0;
    ctx->t_update = ctx->t_bsolve = 0.0;
    ctx->n_update = 0;
    ap_status status = AP_ERR_NOT_CONVERGED;
    const bool low_precision = ctx->o.precision != AP_FP32;
    // relative column residuals from the column norms in rn, and the stop rule
    auto rel_from = [&](double* out) -> bool {
        double fr = 0.0, fb = 0.0;
        for (int k = 0; k < c; ++k) {
            out[k] = bn[k] > 0.0 ? sqrt(rn[k] / bn[k]) : sqrt(rn[k]);
            fr += rn[k];
            fb += bn[k];
        }
        return epoch >= ctx->o.min_epochs && stop_met(ctx->o.stop, ctx->o.tol, c, out, sqrt(fr), sqrt(fb));
    };
    // true residual (in the stopping rule's measure) at the start and after the
    // last refinement: the reference for the escalation test
    rel_from(rel_true);
    double true_prev = rule_measure(ctx->o.stop, c, rel_true, bn);
    AP_CK(cudaEventRecord(ctx->ev_a, ctx->st));
    while (true) {
        int64_t ns = ctx->m;
        if (ctx->o.max_steps > 0) ns = std::min<int64_t>(ns, ctx->o.max_steps - steps);
        if (ns <= 0) break;
        PhaseRange epoch_range(ctx->tc_steps ? "ap: epoch (tensor-core update)" : "ap: epoch (FP32 update)");
        AP_TRY(run_epoch(ctx, ns));
        steps += ns;
        ++epoch;
        if (ctx->tc && !ctx->tc_steps) ++fp32_epochs;
        int nanf = 0, tcerr = 0;
        AP_CK(cudaMemcpyAsync(rn, ctx->colnorm, sizeof(double) * Cp, cudaMemcpyDeviceToHost, ctx->st));
        AP_CK(cudaMemcpyAsync(&nanf, ctx->nan_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        AP_CK(cudaMemcpyAsync(&tcerr, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        AP_CK(cudaStreamSynchronize(ctx->st));
        collect_profile(ctx, ns);
        if (tcerr) {
            status = AP_ERR_TIMEOUT;
            break;
        }
        bool met = rel_from(rel);
        // Divergence of the low-precision updates (their kernel-entry error can
        // exceed what sigma^2 keeps positive definite: large n, small noise,
        // smooth kernels): a NaN, or a tracked residual above twice the last
        // certified one.  Roll W back to the last checkpoint, recompute R and
        // continue with the FP32 update.
        if (ctx->tc_steps && ctx->o.escalate && (nanf || !(rule_measure(ctx->o.stop, c, rel, bn) <= 2.0 * true_prev))) {
            ctx->tc_steps = false;
            drop_graph(ctx);
            AP_CK(cudaMemcpyAsync(ctx->W, ctx->W_ckpt, sizeof(float) * ctx->n * Cp, cudaMemcpyDeviceToDevice, ctx->st));
            AP_CK(cudaMemsetAsync(ctx->nan_flag, 0, sizeof(int), ctx->st));
            AP_CK(cudaEventRecord(ctx->ev_r0, ctx->st));
            AP_TRY(launch_full_residual(ctx, ctx->Bp, ctx->W, ctx->R, kEpiBlockNorms | kEpiColNorms));
            AP_CK(cudaEventRecord(ctx->ev_r1, ctx->st));
            AP_CK(cudaMemcpyAsync(rn, ctx->colnorm, sizeof(double) * Cp, cudaMemcpyDeviceToHost, ctx->st));
            AP_CK(cudaMemcpyAsync(&nanf, ctx->nan_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
            AP_CK(cudaStreamSynchronize(ctx->st));
            float rms = 0.f;
            cudaEventElapsedTime(&rms, ctx->ev_r0, ctx->ev_r1);
            t_refine += rms * 1e-3;
            ++refinements;
            ++ctx->divergences;
            met = rel_from(rel);
            have_true = true;
            true_epoch = epoch;
            for (int k = 0; k < c; ++k) rel_true[k] = rel[k];
            true_prev = rule_measure(ctx->o.stop, c, rel, bn);
        }
        if (nanf) {
            status = AP_ERR_NAN;
            break;
        }
        const bool periodic = ctx->tc_steps && ctx->o.refine_every > 0 && epoch % ctx->o.refine_every == 0;
        if (met || periodic) {
            // Refinement / certification: recompute R = B - K_hat W over all n^2
            // entries in the FP32 form (residual lemma, App. B) and continue
            // from it; the stopping rule is judged on the recomputed residual.
            AP_CK(cudaEventRecord(ctx->ev_r0, ctx->st));
            AP_TRY(launch_full_residual(ctx, ctx->Bp, ctx->W, ctx->R, kEpiBlockNorms | kEpiColNorms));
            AP_CK(cudaEventRecord(ctx->ev_r1, ctx->st));
            AP_CK(cudaMemcpyAsync(rn, ctx->colnorm, sizeof(double) * Cp, cudaMemcpyDeviceToHost, ctx->st));
            AP_CK(cudaMemcpyAsync(&nanf, ctx->nan_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
            AP_CK(cudaStreamSynchronize(ctx->st));
            float rms = 0.f;
            cudaEventElapsedTime(&rms, ctx->ev_r0, ctx->ev_r1);
            t_refine += rms * 1e-3;
            ++refinements;
            if (nanf) {
                status = AP_ERR_NAN;
                break;
            }
            const double tracked_now = rule_measure(ctx->o.stop, c, rel, bn);
            const bool tracked_met = met;
            met = rel_from(rel_true);
            have_true = true;
            true_epoch = epoch;
            // The tracked rule held but the plain FP32 recompute does not confirm
            // it: when K_hat |W| is much larger than B the FP32 sums' own error can
            // exceed tol, so AP_RESID_AUTO certifies with the compensated recompute
            // from here on (refinement then continues from an accurate residual)
            if (tracked_met && !met && !ctx->comp_used && ctx->o.residual_mode == AP_RESID_AUTO)
                ctx->comp_auto = true;
            // Escalation: when the true residual fell by less than half of what
            // the tracked one claims since the last recompute, the low-precision
            // updates' own error, not AP's rate, limits progress
            const double true_now = rule_measure(ctx->o.stop, c, rel_true, bn);
            if (!met && ctx->tc_steps && ctx->o.escalate && true_prev - true_now < 0.5 * (true_prev - tracked_now)) {
                ctx->tc_steps = false;
                drop_graph(ctx);
            }
            if (ctx->tc_steps && true_now <= true_prev)
                AP_CK(cudaMemcpyAsync(ctx->W_ckpt, ctx->W, sizeof(float) * ctx->n * Cp, cudaMemcpyDeviceToDevice,
                                      ctx->st));
            true_prev = true_now;
            for (int k = 0; k < c; ++k) rel[k] = rel_true[k];
        }
        if (met) {
            status = AP_OK;
            break;
        }
        if (epoch >= ctx->o.max_epochs) break;
        if (ctx->o.max_steps > 0 && steps >= ctx->o.max_steps) break;
        if (ctx->o.cancel && *ctx->o.cancel) {
            status = AP_ERR_CANCELLED;
            break;
        }
    }
    // A low-precision run that stopped on its epoch cap reports the true
    // residual of the W it returns: one more FP32 recompute (max_steps runs,
    // used to replay individual steps, are left untouched).
    if (low_precision && status == AP_ERR_NOT_CONVERGED && ctx->o.max_steps <= 0 && epoch > 0 &&
        true_epoch != epoch) {
        AP_CK(cudaEventRecord(ctx->ev_r0, ctx->st));
        AP_TRY(launch_full_residual(ctx, ctx->Bp, ctx->W, ctx->R, kEpiColNorms));
        AP_CK(cudaEventRecord(ctx->ev_r1, ctx->st));
        AP_CK(cudaMemcpyAsync(rn, ctx->colnorm, sizeof(double) * Cp, cudaMemcpyDeviceToHost, ctx->st));
        AP_CK(cudaStreamSynchronize(ctx->st));
        float rms = 0.f;
        cudaEventElapsedTime(&rms, ctx->ev_r0, ctx->ev_r1);
        t_refine += rms * 1e-3;
        ++refinements;
        rel_from(rel_true);
        have_true = true;
    }
    AP_CK(cudaEventRecord(ctx->ev_b, ctx->st));
    AP_CK(launch_unpad_copy(ctx->W, ctx->n, Cp, W_dev, c, ctx->st));
    ++ctx->launches;
    AP_TRY(leave(ctx));
    ctx->r_tracked_c = c;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b);
    if (ctx->o.block_trace && ctx->o.trace_cap > 0) {
        const int64_t k = std::min<int64_t>(steps, ctx->o.trace_cap);
        if (k > 0)
            AP_CK(cudaMemcpy(ctx->o.block_trace, ctx->trace, sizeof(int) * k, cudaMemcpyDeviceToHost));
    }
    if (info) {
        info->epochs = epoch;
        info->steps = steps;
        info->refinements = refinements;
        info->bad_block = -1;
        info->c = c;
        for (int k = 0; k < AP_MAX_RHS; ++k) {
            info->rel_res_tracked[k] = k < c ? rel[k] : 0.0;
            info->rel_res_true[k] = k < c ? (have_true ? rel_true[k] : rel[k]) : 0.0;
        }
        info->t_cache_s = ctx->t_cache;
        info->t_solve_s = ms * 1e-3;
        info->t_refine_s = t_refine;
        info->kernel_entries = (double)steps * (double)ctx->n * ((double)ctx->n / (double)ctx->m) +
                               (double)refinements * (double)ctx->n * (double)ctx->n;
        info->entries_per_s = info->t_solve_s > 0 ? info->kernel_entries / info->t_solve_s : 0.0;
        info->gpu_launches = ctx->launches - l0;
        info->data_fit = 0.0;
        info->t_update_s = ctx->t_update;
        info->n_update = ctx->n_update;
        info->t_blocksolve_s = ctx->t_bsolve;
        info->fp32_epochs = fp32_epochs;
        info->compensated = ctx->comp_used && have_true ? 1 : 0;
        info->diverged = ctx->divergences;
    }
    return status;
}

}  // namespace

namespace ap {

void ctx_grad_view(const ap_ctx* ctx, GradView* v) {
    v->device = ctx->device;
    v->Xs = ctx->Xs;
    v->n = ctx->n;
    v->d = ctx->d;
    v->D = ctx->D;
    v->kernel = ctx->kernel;
    v->s = ctx->s;
    v->ell = ctx->ell;
    v->stream = ctx->ust;
}

void grad_finish(const GradView& v, const double* raw, double* out_host) {
    const double fac = v.kernel == AP_RBF ? 2.0 / 1.4426950408889634 : (v.kernel == AP_MATERN32 ? 1.0 : 1.0 / 3.0);
    for (int k = 0; k < v.d; ++k) out_host[k] = (double)v.s * fac * raw[k] / (double)v.ell[k];
    out_host[v.d] = raw[v.D];
    out_host[v.d + 1] = raw[v.D + 1];
}

#ifdef AP_CHECKED
namespace {
struct ChkUnit {
    const char* unit;
    unsigned int (*read_and_clear)();
};
std::vector<ChkUnit>& chk_units() {
    static std::vector<ChkUnit> units;
    return units;
}
}  // namespace

int chk_register(const char* unit, unsigned int (*read_and_clear)()) {
    chk_units().push_back({unit, read_and_clear});
    return 1;
}
#endif

}  // namespace ap

extern "C" {

int32_t ap_bounds_violations(char* where, int32_t cap) {
#ifdef AP_CHECKED
    cudaDeviceSynchronize();
    int32_t count = 0;
    for (const ap::ChkUnit& u : ap::chk_units()) {
        const unsigned int line = u.read_and_clear();
        if (!line) continue;
        if (count == 0 && where && cap > 0) {
            const char* base = strrchr(u.unit, '/');
            snprintf(where, (size_t)cap, "%s:%u", base ? base + 1 : u.unit, line);
        }
        ++count;
    }
    return count;
#else
    (void)where;
    (void)cap;
    return -1;
#endif
}

void ap_opts_default(ap_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->block = 4096;
    o->select = AP_SEL_GS;
    o->stop = AP_STOP_MEAN_REL;
    o->tol = 1.0;
    o->min_epochs = 11;
    o->max_epochs = 1000;
    o->max_steps = 0;
    o->precision = AP_FP32;
    o->refine_every = 4;
    o->seed = 0;
    o->stream = nullptr;
    o->hbm_budget = 0;
    o->block_trace = nullptr;
    o->trace_cap = 0;
    o->profile = 0;
    o->residual_mode = AP_RESID_AUTO;
    o->cache_gemm = AP_CACHE_TC_EXACT;
    o->wait_limit_cycles = 0;
    o->cancel = nullptr;
    o->escalate = 1;
}

size_t ap_sizeof_opts(void) { return sizeof(ap_opts); }
size_t ap_sizeof_info(void) { return sizeof(ap_info); }
size_t ap_sizeof_hyper(void) { return sizeof(ap_hyper); }

const char* ap_status_str(ap_status s) {
    switch (s) {
        case AP_OK: return "AP_OK";
        case AP_ERR_INVALID_ARG: return "AP_ERR_INVALID_ARG";
        case AP_ERR_NOMEM: return "AP_ERR_NOMEM";
        case AP_ERR_NOT_SPD: return "AP_ERR_NOT_SPD";
        case AP_ERR_NAN: return "AP_ERR_NAN";
        case AP_ERR_NOT_CONVERGED: return "AP_ERR_NOT_CONVERGED";
        case AP_ERR_TIMEOUT: return "AP_ERR_TIMEOUT";
        case AP_ERR_CUDA: return "AP_ERR_CUDA";
        case AP_ERR_UNSUPPORTED: return "AP_ERR_UNSUPPORTED";
        case AP_ERR_SCRATCH_LIMIT: return "AP_ERR_SCRATCH_LIMIT";
        case AP_ERR_CANCELLED: return "AP_ERR_CANCELLED";
    }
    return "AP_ERR_UNKNOWN";
}

ap_status ap_create(ap_ctx** out, const float* X_dev, int64_t n, int32_t d, const ap_hyper* h, const ap_opts* o) {
    if (!out) return AP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!X_dev || n < 1 || d < 1 || d > AP_MAX_DIM || !o) return AP_ERR_INVALID_ARG;
    AP_TRY(check_hyper(h, d));
    if (o->block < 1 || o->select < 0 || o->select > 2 || o->stop < 0 || o->stop > 3) return AP_ERR_INVALID_ARG;
    if (o->precision < 0 || o->precision > 2 || o->max_epochs < 1 || o->min_epochs < 0) return AP_ERR_INVALID_ARG;
    if (o->residual_mode < 0 || o->residual_mode > 2) return AP_ERR_INVALID_ARG;
    if (o->cache_gemm < 0 || o->cache_gemm > 1) return AP_ERR_INVALID_ARG;
    if (o->precision == AP_FP16_REFINE) return AP_ERR_UNSUPPORTED;
    if (o->precision == AP_BF16_REFINE && d + 2 > 32) return AP_ERR_UNSUPPORTED;
    ap_ctx* ctx = new (std::nothrow) ap_ctx();
    if (!ctx) return AP_ERR_NOMEM;
    ctx->n = n;
    ctx->d = d;
    ctx->D = pad_d(d);
    ctx->X = X_dev;
    ctx->o = *o;
    copy_hyper(ctx, h);
    ctx->b = std::min<int64_t>(o->block, n);
    ctx->m = (n + ctx->b - 1) / ctx->b;
    ctx->nt = (int)((ctx->b + kTile - 1) / kTile);
    ctx->ntri = (int64_t)ctx->nt * (ctx->nt + 1) / 2;
    ctx->ust = (cudaStream_t)o->stream;
    ctx->tc = o->precision == AP_BF16_REFINE;
    ctx->kd = tc_kd(d);
    ctx->cpb = tc_chunks_per_block(ctx->b);
    ctx->tps128 = (ctx->b + 127) / 128;
    {
        int sms = 0;
        if (cudaGetDevice(&ctx->device) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return AP_ERR_CUDA;
        }
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess && sms > 0)
            ctx->num_sms = sms;
        cudaGetLastError();
    }
    ap_status s = AP_OK;
    auto fail = [&](ap_status e) {
        free_all(ctx);
        delete ctx;
        return e;
    };
    if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&ctx->ev_a) != cudaSuccess || cudaEventCreate(&ctx->ev_b) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_sync, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&ctx->ev_r0) != cudaSuccess || cudaEventCreate(&ctx->ev_r1) != cudaSuccess) {
        cudaGetLastError();
        return fail(AP_ERR_CUDA);
    }
    if ((s = dalloc_t(ctx, &ctx->Xs, (size_t)(n * ctx->D))) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->Xs_lo, (size_t)(n * ctx->D))) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->norms, (size_t)ctx->m)) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->colnorm, AP_MAX_RHS)) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->gout, AP_MAX_DIM + 4)) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->ticket, 4)) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->sel, 1)) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->step, 1)) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->nan_flag, 1)) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->bad, (size_t)ctx->m)) != AP_OK) return fail(s);
    if ((s = dalloc_t(ctx, &ctx->tc_err, 1)) != AP_OK) return fail(s);
    if (ctx->tc) {
        if ((s = dalloc_t(ctx, &ctx->XA, tc_rows_bytes(ctx->m * ctx->tps128, ctx->kd))) != AP_OK) return fail(s);
        if ((s = dalloc_t(ctx, &ctx->XB, tc_cols_bytes(ctx->m, ctx->cpb, ctx->kd))) != AP_OK) return fail(s);
        if ((s = dalloc_t(ctx, &ctx->tc_scr, tc_share_bytes(ctx->num_sms, AP_MAX_RHS) / sizeof(float))) != AP_OK)
            return fail(s);
        if ((s = dalloc_t(ctx, &ctx->tc_tick, (size_t)ctx->num_sms)) != AP_OK) return fail(s);
        if (cudaMemsetAsync(ctx->tc_tick, 0, sizeof(int) * ctx->num_sms, ctx->st) != cudaSuccess) {
            cudaGetLastError();
            return fail(AP_ERR_CUDA);
        }
    }
    if (cudaMemsetAsync(ctx->ticket, 0, 4 * sizeof(unsigned), ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->sel, 0, sizeof(int), ctx->st) != cudaSuccess) {
        cudaGetLastError();
        return fail(AP_ERR_CUDA);
    }
    if (o->profile) {
        ctx->ev_bs.resize((size_t)(2 * ctx->m), nullptr);
        ctx->ev_up.resize((size_t)(2 * ctx->m), nullptr);
        for (size_t k = 0; k < ctx->ev_bs.size(); ++k)
            if (cudaEventCreate(&ctx->ev_bs[k]) != cudaSuccess || cudaEventCreate(&ctx->ev_up[k]) != cudaSuccess) {
                cudaGetLastError();
                return fail(AP_ERR_CUDA);
            }
    }
    if ((s = enter(ctx)) != AP_OK) return fail(s);
    s = build_cache(ctx);
    if (s != AP_OK) return fail(s);
    *out = ctx;
    return AP_OK;
}

ap_status ap_set_hyper(ap_ctx* ctx, const ap_hyper* h) {
    if (!ctx) return AP_ERR_INVALID_ARG;
    AP_DEVICE_GUARD(ctx);
    AP_TRY(check_hyper(h, ctx->d));
    if (h->kernel != ctx->kernel) return AP_ERR_INVALID_ARG;
    copy_hyper(ctx, h);
    AP_TRY(enter(ctx));
    return build_cache(ctx);
}

ap_status ap_solve(ap_ctx* ctx, const float* B_dev, int32_t c, const float* W0_dev, float* W_dev, ap_info* info) {
    if (!ctx || !B_dev || !W_dev || c < 1 || c > AP_MAX_RHS) return AP_ERR_INVALID_ARG;
    AP_DEVICE_GUARD(ctx);
    ap_status s = solve_impl(ctx, B_dev, c, W0_dev, W_dev, info);
    if (info && s != AP_OK) info->bad_block = -1;
    return s;
}

ap_status ap_solve_host(const float* X_host, int64_t n, int32_t d, const ap_hyper* h, const ap_opts* o,
                        const float* B_host, int32_t c, float* W_host, ap_info* info) {
    if (!X_host || !B_host || !W_host || !h || !o || n < 1 || d < 1 || d > AP_MAX_DIM || c < 1 || c > AP_MAX_RHS)
        return AP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)o->stream;
    const size_t xb = sizeof(float) * (size_t)n * (size_t)d, bb = sizeof(float) * (size_t)n * (size_t)c;
    float *X = nullptr, *B = nullptr, *W = nullptr;
    auto release = [&]() {
        cudaFreeAsync(X, st);
        cudaFreeAsync(B, st);
        cudaFreeAsync(W, st);
        cudaStreamSynchronize(st);
        cudaGetLastError();
    };
    if (cudaMallocAsync((void**)&X, xb, st) != cudaSuccess || cudaMallocAsync((void**)&B, bb, st) != cudaSuccess ||
        cudaMallocAsync((void**)&W, bb, st) != cudaSuccess) {
        release();
        return AP_ERR_NOMEM;
    }
    if (cudaMemcpyAsync(X, X_host, xb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(B, B_host, bb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        release();
        return AP_ERR_CUDA;
    }
    ap_ctx* ctx = nullptr;
    ap_status s = ap_create(&ctx, X, n, d, h, o);
    if (s != AP_OK) {
        release();
        return s;
    }
    s = ap_solve(ctx, B, c, nullptr, W, info);
    const bool wrote = s == AP_OK || s == AP_ERR_NOT_CONVERGED || s == AP_ERR_CANCELLED;
    if (wrote && (cudaMemcpyAsync(W_host, W, bb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                  cudaStreamSynchronize(st) != cudaSuccess))
        s = AP_ERR_CUDA;
    ap_destroy(ctx);
    release();
    return s;
}

ap_status ap_residual(ap_ctx* ctx, const float* B_dev, int32_t c, const float* W_dev, float* R_dev) {
    if (!ctx || !B_dev || !W_dev || !R_dev || c < 1 || c > AP_MAX_RHS) return AP_ERR_INVALID_ARG;
    AP_DEVICE_GUARD(ctx);
    const int Cp = pad_c(c);
    AP_TRY(ensure_solve(ctx, Cp));
    ctx->r_tracked_c = 0;
    AP_TRY(enter(ctx));
    AP_CK(launch_pad_copy(B_dev, ctx->n, c, ctx->Bp, Cp, ctx->st));
    AP_CK(launch_pad_copy(W_dev, ctx->n, c, ctx->Tmp, Cp, ctx->st));
    ctx->launches += 2;
    AP_TRY(launch_full_residual(ctx, ctx->Bp, ctx->Tmp, ctx->R, 0));
    AP_CK(launch_unpad_copy(ctx->R, ctx->n, Cp, R_dev, c, ctx->st));
    ++ctx->launches;
    return leave(ctx);
}

ap_status ap_predict_mean(ap_ctx* ctx, const float* w_dev, const float* Xs_dev, int64_t M, float* mean_dev) {
    PhaseRange range("ap: posterior mean");
    if (!ctx || !w_dev || !Xs_dev || !mean_dev || M < 1) return AP_ERR_INVALID_ARG;
    AP_DEVICE_GUARD(ctx);
    if (M > ctx->Xt_alloc) {
        dfree(ctx, ctx->Xt);
        ctx->Xt_alloc = 0;
        AP_TRY(dalloc_t(ctx, &ctx->Xt, (size_t)(M * ctx->D)));
        ctx->Xt_alloc = M;
    }
    AP_TRY(enter(ctx));
    AP_CK(cudaMemsetAsync(ctx->nan_flag, 0, sizeof(int), ctx->st));
    AP_TRY(prep_inputs(ctx, Xs_dev, M, ctx->Xt, nullptr));
    const int64_t rows = kmv_rows_per_cta(ctx->D, 1);
    Shape sh;
    sh.rows = rows;
    sh.tps = (M + rows - 1) / rows;
    sh.ntiles = sh.tps;
    sh.S = choose_split(sh.ntiles, ctx->n);
    KmvParams kp = {};
    kp.Xa = ctx->Xt;
    kp.na = M;
    kp.Xb = ctx->Xs;
    kp.nb = ctx->n;
    kp.V = w_dev;
    kp.base = nullptr;
    kp.base_const = ctx->mean;
    kp.out = mean_dev;
    kp.sgn = 1.f;
    kp.s = ctx->s;
    kp.noise = 0.f;
    kp.noise_diag = 0;
    kp.col0 = 0;
    kp.ncols = ctx->n;
    kp.epi = make_epi(ctx, 0, 0, sh);
    kp.epi.seg = M;
    AP_CK(launch_kmv(ctx->kernel, kp, ctx->D, 1, ctx->st));
    ++ctx->launches;
    int nanx = 0;
    AP_CK(cudaMemcpyAsync(&nanx, ctx->nan_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    AP_TRY(leave(ctx));
    return nanx ? AP_ERR_NAN : AP_OK;
}

static ap_status grad_quadforms_impl(ap_ctx* ctx, const float* U, const float* V, int Cp, const double* alpha,
                                     int c, double* out_host) {
    const int64_t rows = grad_rows_per_cta(ctx->D, Cp);
    const int64_t ntiles = (ctx->n + rows - 1) / rows;
    const int S = choose_split(ntiles, ctx->n);
    const int NA = ctx->D + 2;
    const int64_t need = std::max<int64_t>(ntiles * S * NA, 256);
    if (need > ctx->gpart_alloc) {
        dfree(ctx, ctx->gpart);
        ctx->gpart_alloc = 0;
        AP_TRY(dalloc_t(ctx, &ctx->gpart, (size_t)need));
        ctx->gpart_alloc = need;
    }
    GradParams gp = {};
    gp.Xs = ctx->Xs;
    gp.n = ctx->n;
    gp.U = U;
    gp.V = V;
    for (int k = 0; k < c; ++k) gp.alpha[k] = (float)alpha[k];
    gp.ntiles = ntiles;
    gp.S = S;
    gp.part = ctx->gpart;
    gp.ticket = ctx->ticket + 1;
    gp.out = ctx->gout;
    AP_CK(launch_grad(ctx->kernel, gp, ctx->D, Cp, ctx->st));
    ++ctx->launches;
    double raw[AP_MAX_DIM + 2] = {};
    AP_CK(cudaMemcpyAsync(raw, ctx->gout, sizeof(double) * NA, cudaMemcpyDeviceToHost, ctx->st));
    AP_CK(cudaStreamSynchronize(ctx->st));
    const double fac = ctx->kernel == AP_RBF ? 2.0 / 1.4426950408889634 : (ctx->kernel == AP_MATERN32 ? 1.0 : 1.0 / 3.0);
    for (int k = 0; k < ctx->d; ++k) out_host[k] = (double)ctx->s * fac * raw[k] / (double)ctx->ell[k];
    out_host[ctx->d] = raw[ctx->D];
    out_host[ctx->d + 1] = raw[ctx->D + 1];
    return AP_OK;
}

ap_status ap_grad_quadforms(ap_ctx* ctx, const float* U_dev, const float* V_dev, int32_t c, const double* alpha_host,
                            double* out_host) {
    PhaseRange range("ap: gradient quadratic forms");
    if (!ctx || !U_dev || !V_dev || !alpha_host || !out_host || c < 1 || c > AP_MAX_RHS) return AP_ERR_INVALID_ARG;
    AP_DEVICE_GUARD(ctx);
    const int Cp = pad_c(c);
    AP_TRY(ensure_solve(ctx, Cp));
    AP_TRY(enter(ctx));
    AP_CK(launch_pad_copy(U_dev, ctx->n, c, ctx->Tmp, Cp, ctx->st));
    AP_CK(launch_pad_copy(V_dev, ctx->n, c, ctx->Bp, Cp, ctx->st));
    ctx->launches += 2;
    AP_TRY(grad_quadforms_impl(ctx, ctx->Tmp, ctx->Bp, Cp, alpha_host, c, out_host));
    return leave(ctx);
}

ap_status ap_mll_grad(ap_ctx* ctx, const float* y_dev, int32_t n_probes, const float* Z_dev, float* grad_host,
                      ap_info* info) {
    PhaseRange range("ap: MLL gradient");
    if (!ctx || !y_dev || !grad_host || n_probes < 0 || n_probes + 1 > AP_MAX_RHS) return AP_ERR_INVALID_ARG;
    AP_DEVICE_GUARD(ctx);
    const int l = n_probes, c = l + 1;
    float* Bfull = nullptr;
    float* Wfull = nullptr;
    AP_TRY(dalloc_t(ctx, &Bfull, (size_t)(ctx->n * c)));
    ap_status s = dalloc_t(ctx, &Wfull, (size_t)(ctx->n * c));
    if (s != AP_OK) {
        dfree(ctx, Bfull);
        return s;
    }
    auto done = [&](ap_status e) {
        dfree(ctx, Bfull);
        dfree(ctx, Wfull);
        return e;
    };
    if ((s = enter(ctx)) != AP_OK) return done(s);
    if (launch_assemble_rhs(y_dev, ctx->mean, Z_dev, l, ctx->o.seed, ctx->n, Bfull, nullptr, ctx->st) != cudaSuccess)
        return done(AP_ERR_CUDA);
    ++ctx->launches;
    const int64_t l0 = ctx->launches;
    ap_status st = solve_impl(ctx, Bfull, c, nullptr, Wfull, info);
    if (st != AP_OK && st != AP_ERR_NOT_CONVERGED) return done(st);
    // U = W (padded, in ctx->W), V = [u, z_1..z_l]
    const int Cp = ctx->Cp;
    if (launch_assemble_v(ctx->W, Cp, Bfull, c, ctx->n, ctx->Tmp, ctx->st) != cudaSuccess) return done(AP_ERR_CUDA);
    ++ctx->launches;
    double alpha[AP_MAX_RHS] = {};
    alpha[0] = -0.5;
    for (int k = 1; k < c; ++k) alpha[k] = 0.5 / (double)l;
    double g[AP_MAX_DIM + 2] = {};
    if ((s = grad_quadforms_impl(ctx, ctx->W, ctx->Tmp, Cp, alpha, c, g)) != AP_OK) return done(s);
    if (launch_dot0(ctx->W, Cp, nullptr, 0, ctx->n, ctx->gpart, ctx->ticket + 2, ctx->gout, ctx->st) != cudaSuccess ||
        launch_dot0(ctx->W, Cp, Bfull, c, ctx->n, ctx->gpart, ctx->ticket + 2, ctx->gout + 1, ctx->st) != cudaSuccess)
        return done(AP_ERR_CUDA);
    ctx->launches += 2;
    double dots[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(dots, ctx->gout, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess)
        return done(AP_ERR_CUDA);
    if ((s = leave(ctx)) != AP_OK) return done(s);
    const double usum = dots[0];
    if (info) info->data_fit = 0.5 * dots[1];
    for (int k = 0; k < ctx->d + 2; ++k) grad_host[k] = (float)g[k];
    grad_host[ctx->d + 2] = (float)(-usum);
    if (info) info->gpu_launches += ctx->launches - l0;
    return done(st);
}

int64_t ap_launch_count(const ap_ctx* ctx) { return ctx ? ctx->launches : 0; }

int32_t ap_last_cuda_error(const ap_ctx* ctx) { return ctx ? (int32_t)ctx->last_cuda : 0; }

size_t ap_device_bytes(const ap_ctx* ctx) { return ctx ? ctx->bytes : 0; }

ap_status ap_tracked_residual(ap_ctx* ctx, int32_t c, float* R_dev) {
    if (!ctx || !R_dev || c < 1 || c > AP_MAX_RHS) return AP_ERR_INVALID_ARG;
    if (ctx->r_tracked_c != c || !ctx->R) return AP_ERR_INVALID_ARG;
    AP_DEVICE_GUARD(ctx);
    AP_TRY(enter(ctx));
    AP_CK(launch_unpad_copy(ctx->R, ctx->n, ctx->Cp, R_dev, c, ctx->st));
    ++ctx->launches;
    return leave(ctx);
}

ap_status ap_phi_fp64_eval(int32_t kernel, const double* r2_host, int64_t count, double* phi_host) {
    if (kernel < AP_RBF || kernel > AP_MATERN52 || count < 0) return AP_ERR_INVALID_ARG;
    if (count == 0) return AP_OK;
    if (!r2_host || !phi_host) return AP_ERR_INVALID_ARG;
    const size_t bytes = sizeof(double) * (size_t)count;
    double* d_r2 = nullptr;
    double* d_out = nullptr;
    if (cudaMalloc(&d_r2, bytes) != cudaSuccess || cudaMalloc(&d_out, bytes) != cudaSuccess) {
        cudaFree(d_r2);
        cudaGetLastError();
        return AP_ERR_NOMEM;
    }
    cudaError_t err = cudaMemcpy(d_r2, r2_host, bytes, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = launch_phi_fp64_eval(kernel, d_r2, count, d_out, 0);
    if (err == cudaSuccess) err = cudaMemcpy(phi_host, d_out, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d_r2);
    cudaFree(d_out);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return AP_ERR_CUDA;
    }
    return AP_OK;
}

void ap_destroy(ap_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard dg(ctx->device);
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    free_all(ctx);
    delete ctx;
}

}  // extern "C"
