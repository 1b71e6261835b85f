/*
 * ap.h -- C ABI of the GB300 alternating-projection (AP) solver for Gaussian
 * process kernel systems (K_hat) W = B, K_hat = s * k_l(X, X) + sigma^2 I.
 *
 * The method is Alg. 1 of Wu et al., "Large-Scale Gaussian Processes via
 * Alternating Projection" (AISTATS 2024): per inner step select a block I by
 * the modified Gauss-Southwell rule (Eq. approximate_gauss_southwell), solve
 * Delta = K_II^{-1} R_I with the cached Cholesky factor of K_II (Sec. 3,
 * "Cached Cholesky Factors"), then W_I += Delta (Eq. text_update_of_w) and
 * R -= K_hat(X, X_I) Delta (Eq. text_update_of_r), the kernel block evaluated
 * on the fly and never stored.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major.  X is n x d, B, W0, W, R are n x c, all FP32.
 *     Pointers named *_dev are device pointers, *_host host pointers.
 *   - The caller owns every buffer it passes.  X must stay alive and unchanged
 *     for the life of the context (it is read again by ap_set_hyper).  The
 *     context owns its scaled copy of X, the Cholesky cache and its work
 *     buffers, and frees them in ap_destroy.
 *   - Work is enqueued on opts.stream (a cudaStream_t, NULL = legacy stream),
 *     and every call returns only once its results are in the caller's
 *     buffers.
 *   - Errors come back as ap_status codes; nothing exits, traps or prints.
 *     After AP_ERR_CUDA the context should be destroyed.
 *   - A context is not thread safe: one call at a time per context.
 *   - A context belongs to the device that was current at ap_create.  Every
 *     call makes that device current for its duration and restores the
 *     caller's current device before it returns.
 */
#ifndef AP_H
#define AP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AP_MAX_RHS 32 /* largest c (1 label column + up to 31 probes) */
#define AP_MAX_DIM 32 /* largest input dimension d */

typedef enum {
    AP_OK = 0,
    AP_ERR_INVALID_ARG = 1,   /* a size, pointer or option is out of range */
    AP_ERR_NOMEM = 2,         /* device allocation failed, or over opts.hbm_budget */
    AP_ERR_NOT_SPD = 3,       /* a diagonal block K_II failed Cholesky: info.bad_block */
    AP_ERR_NAN = 4,           /* a NaN or Inf appeared in the residual */
    AP_ERR_NOT_CONVERGED = 5, /* max_epochs / max_steps reached; W and info still written */
    AP_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (serving workers) */
    AP_ERR_CUDA = 7,          /* a CUDA runtime call failed */
    AP_ERR_UNSUPPORTED = 8,   /* option combination not built */
    AP_ERR_SCRATCH_LIMIT = 9, /* ap_grad_quadforms_static: problem exceeds the fixed scratch */
    AP_ERR_CANCELLED = 10     /* the caller's cancel flag was set (checked between epochs) */
} ap_status;

/* Kernel family, Sec. 5 ("Datasets and Models") and App. E (Matern nu = 1.5):
 * k(x, x') = s * phi(r), r = ||(x - x') / l|| (ARD lengthscales l),
 *   AP_RBF:      phi = exp(-r^2 / 2)
 *   AP_MATERN32: phi = (1 + sqrt(3) r) exp(-sqrt(3) r)
 *   AP_MATERN52: phi = (1 + sqrt(5) r + 5 r^2 / 3) exp(-sqrt(5) r)
 * The noise sigma^2 is added on the index diagonal only (sigma^2 I). */
typedef enum { AP_RBF = 0, AP_MATERN32 = 1, AP_MATERN52 = 2 } ap_kernel;

/* Arithmetic of the residual update.
 *   AP_FP32:         kernel blocks and contraction in FP32 (SIMT).
 *   AP_BF16_REFINE:  kernel blocks and K*Delta on tensor cores with BF16
 *                    operands and FP32 accumulation; accuracy recovered by
 *                    recomputing R = B - K_hat W in the FP32 form (iterative
 *                    refinement, justified by the residual lemma of App. B).
 *   AP_FP16_REFINE:  reserved; ap_create returns AP_ERR_UNSUPPORTED.  One FP16
 *                    product (11-bit kernel values) perturbs K_hat by about
 *                    2^-12 sqrt(n) max|K_ij| in norm, which exceeds sigma^2 at
 *                    the sizes this library targets (n = 262,144, sigma^2 =
 *                    1e-2), so the perturbed operator is not positive definite
 *                    and the iteration diverges. */
typedef enum { AP_FP32 = 0, AP_BF16_REFINE = 1, AP_FP16_REFINE = 2 } ap_precision;

/* Block selection (Sec. 3, "Block Selection"): Gauss-Southwell on
 * ||R_{I,:}||_F^2 (ties to the smallest block), cyclic (step j picks block
 * j mod m), or uniform random (counter-based SplitMix64 of (seed, step)). */
typedef enum { AP_SEL_GS = 0, AP_SEL_CYCLIC = 1, AP_SEL_RANDOM = 2 } ap_select;

/* Stopping rule checked after every epoch (Sec. 5, "Alternating Projection
 * Details"): MEAN_REL = average of per-column ||r_i|| / ||b_i|| strictly below
 * tol (the paper's experiments); MAX_REL = every column <= tol; FRO =
 * ||R||_F <= tol ||B||_F (Alg. 1); Y_REL = the first column only <= tol. */
typedef enum { AP_STOP_MEAN_REL = 0, AP_STOP_MAX_REL = 1, AP_STOP_FRO = 2, AP_STOP_Y_REL = 3 } ap_stop;

/* Arithmetic of the full residual recompute R = B - K_hat W (refinement and
 * certification of the stopping rule, and ap_residual):
 *   AP_RESID_AUTO:        compensated when opts.tol <= 1e-5, plain FP32 otherwise,
 *                         switching to compensated for the rest of a solve when the
 *                         tracked residual meets the rule but a plain FP32
 *                         recompute does not confirm it (the FP32 sums' own error,
 *                         about 2^-24 sqrt(n) ||K_hat |W| ||, can exceed tol);
 *   AP_RESID_FP32:        plain FP32 kernel entries and sums;
 *   AP_RESID_COMPENSATED: double-float FP32 (error-free transformations), kernel
 *                         entries to ~1e-11 relative; about 10x the cost. */
typedef enum { AP_RESID_AUTO = 0, AP_RESID_FP32 = 1, AP_RESID_COMPENSATED = 2 } ap_residual_mode;

/* Hyperparameters (Sec. 5): ARD lengthscales (host array of d floats),
 * outputscale s, noise sigma^2 and constant prior mean mu. */
typedef struct ap_hyper {
    ap_kernel kernel;
    int32_t d;
    const float* lengthscale;
    float outputscale;
    float noise;
    float mean;
} ap_hyper;

/* Solver options.  ap_opts_default fills the paper's values: GS selection,
 * MEAN_REL with tol 1 (training), at least 11 and at most 1000 epochs. */
/* Arithmetic of the trailing (SYRK/GEMM) updates of the FP64 block Cholesky
 * (Sec. 3, "Cached Cholesky Factors"), the bulk of its b^3/3 flops per block.
 *   AP_CACHE_TC_EXACT: FP64 matrix, products formed exactly from 7-bit integer
 *                      slices on the BF16 tensor cores and combined in 64-bit
 *                      integers (error-free splitting), so each update has the
 *                      accuracy of an FP64 GEMM.  Default.
 *   AP_CACHE_FP64:     FP64 FMA on the CUDA cores. */
typedef enum { AP_CACHE_TC_EXACT = 0, AP_CACHE_FP64 = 1 } ap_cache_gemm;

typedef struct ap_opts {
    int64_t block;        /* block size b (sequential partition, Sec. 5); last block may be short */
    int32_t select;       /* ap_select */
    int32_t stop;         /* ap_stop */
    double tol;           /* stopping tolerance epsilon */
    int32_t min_epochs;   /* default 11 */
    int32_t max_epochs;   /* default 1000 */
    int64_t max_steps;    /* > 0: stop after this many inner steps in total (bounded runs) */
    int32_t precision;    /* ap_precision */
    int32_t refine_every; /* low-precision forms: recompute R in FP32 every this many epochs */
    uint64_t seed;        /* AP_SEL_RANDOM stream, and probes when ap_mll_grad gets Z_dev = NULL */
    void* stream;         /* cudaStream_t for all work of this context */
    size_t hbm_budget;    /* bytes the context may allocate; 0 = no limit */
    int32_t* block_trace; /* optional host array: chosen block of each step */
    int64_t trace_cap;    /* capacity of block_trace */
    int32_t profile;      /* 1: time every block solve and residual update with CUDA events */
    int32_t residual_mode; /* ap_residual_mode: arithmetic of the residual recompute */
    int32_t cache_gemm;   /* ap_cache_gemm: arithmetic of the Cholesky trailing updates */
    int64_t wait_limit_cycles; /* bound of each device-side wait of the tensor-core update, in SM
                                  clock cycles; <= 0: about 2 s.  A wait that runs out ends the
                                  kernel early and the call returns AP_ERR_TIMEOUT */
    const volatile int32_t* cancel; /* optional host flag: when it reads non-zero at the end of an
                                       epoch, ap_solve / ap_mll_grad stop with AP_ERR_CANCELLED
                                       (W holds the last iterate) */
    int32_t escalate;     /* low-precision forms: 1 (default) = run the remaining epochs with the
                             FP32 update when a refinement finds that the true residual fell by
                             less than half of what the tracked one claims since the previous
                             recompute (the low-precision updates' error, not AP's convergence,
                             limits progress), or when the tracked residual turns NaN or exceeds
                             twice the last certified one (divergence: W is rolled back to the
                             last refinement that lowered the true residual); 0 = never */
} ap_opts;

/* Report of ap_solve / ap_mll_grad.  rel_res_* hold the first c columns. */
typedef struct ap_info {
    int32_t epochs;
    int32_t refinements;
    int64_t steps;
    int32_t bad_block;                    /* AP_ERR_NOT_SPD: first failing block */
    int32_t c;                            /* number of right-hand sides */
    double rel_res_tracked[AP_MAX_RHS];   /* ||R_col|| / ||B_col|| of the tracked residual */
    double rel_res_true[AP_MAX_RHS];      /* the same for B - K_hat W after the last refinement
                                             (low-precision forms); equals tracked for FP32 */
    double t_cache_s;                     /* Cholesky cache build time of the context */
    double t_solve_s;                     /* wall time of the iteration */
    double t_refine_s;                    /* part of t_solve_s spent in refinement passes */
    double kernel_entries;                /* kernel-matrix entries evaluated by the iteration */
    double entries_per_s;                 /* kernel_entries / t_solve_s */
    int64_t gpu_launches;                 /* kernels launched by this call */
    double data_fit;                      /* ap_mll_grad: 1/2 (y - mu)^T u, u = K_hat^{-1}(y - mu) */
    double t_update_s;                    /* opts.profile: summed duration of the residual-update kernels */
    int64_t n_update;                     /* opts.profile: number of residual-update launches timed */
    double t_blocksolve_s;                /* opts.profile: summed duration of the block solves */
    int32_t fp32_epochs;                  /* epochs run with the FP32 update after an escalation */
    int32_t compensated;                  /* rel_res_true comes from the compensated recompute */
    int32_t diverged;                     /* the low-precision updates diverged and were rolled back */
} ap_info;

typedef struct ap_ctx ap_ctx;

/* Fill *o with the defaults: block 4096, GS, MEAN_REL, tol 1, 11..1000 epochs,
 * FP32, refine_every 4, seed 0, default stream, no budget, no trace,
 * escalation on. */
void ap_opts_default(ap_opts* o);

/* Create a solver context for the n training inputs X_dev (device, n x d FP32,
 * borrowed) and build the cached Cholesky factors of every diagonal block
 * K_hat_II (Sec. 3, "Cached Cholesky Factors": factor once per hyperparameter
 * setting; Table 6: (1/3) n b^2 flops, n b memory).  The factorisation runs in
 * FP64; the factor's inverse L_I^{-1} is stored in FP32.
 * Errors: INVALID_ARG (n < 1, d not in [1, 32], block < 1, bad hyper),
 * NAN (a NaN or Inf in X), NOMEM, NOT_SPD, TIMEOUT, CUDA; no context is
 * returned on error. */
ap_status ap_create(ap_ctx** out, const float* X_dev, int64_t n, int32_t d,
                    const ap_hyper* h, const ap_opts* o);

/* Replace the hyperparameters (same kernel family and d) and refactor the cache. */
ap_status ap_set_hyper(ap_ctx* ctx, const ap_hyper* h);

/* Solve K_hat W = B for c in [1, 32] right-hand sides by Alg. 1.  B_dev is
 * n x c (device).  W0_dev (n x c, may be NULL) is a starting point: then R is
 * first recomputed as B - K_hat W0 (warm start / resume).  W_dev (n x c) gets
 * the result.  info (may be NULL) gets the report.
 * Returns OK when the stopping rule held after >= min_epochs epochs,
 * NOT_CONVERGED at max_epochs / max_steps (W still written), NAN (a NaN or Inf
 * in the residual, e.g. from B), CANCELLED (opts.cancel), TIMEOUT (a bounded
 * device wait of the tensor-core update ran out), CUDA. */
ap_status ap_solve(ap_ctx* ctx, const float* B_dev, int32_t c, const float* W0_dev,
                   float* W_dev, ap_info* info);

/* One-shot solve for host-resident data: copies X_host (n x d) and B_host
 * (n x c) to the device, builds the context (ap_create: the Cholesky cache),
 * runs ap_solve (opts as for ap_create/ap_solve; W0 none), copies W to W_host
 * (n x c) and releases everything, all on opts.stream.  Page-locked host
 * buffers give full-bandwidth copies; pageable ones work too.  info (may be
 * NULL) as for ap_solve.  Returns ap_create's or ap_solve's status; W_host is
 * written whenever ap_solve wrote W. */
ap_status ap_solve_host(const float* X_host, int64_t n, int32_t d, const ap_hyper* h, const ap_opts* o,
                        const float* B_host, int32_t c, float* W_host, ap_info* info);

/* True residual R = B - K_hat W (n x c, device), FP32 form, all n^2 kernel
 * entries evaluated on the fly (the residual lemma of App. B).  Used for
 * refinement and certification. */
ap_status ap_residual(ap_ctx* ctx, const float* B_dev, int32_t c, const float* W_dev,
                      float* R_dev);

/* Posterior mean (Sec. 2): mean_dev[t] = mu + s * sum_j phi(x*_t, x_j) w_j for
 * the M test inputs Xs_dev (device, M x d).  w_dev (device, n) is
 * K_hat^{-1} (y - mu), e.g. column 0 of ap_solve's W.  No noise term.
 * AP_ERR_NAN (means still written) when a test input is NaN or Inf. */
ap_status ap_predict_mean(ap_ctx* ctx, const float* w_dev, const float* Xs_dev, int64_t M,
                          float* mean_dev);

/* The fused derivative quadratic forms of Eq. loss_grad_unbiased:
 *   out_host[p] = sum_col alpha_host[col] * U[:,col]^T (dK_hat / dtheta_p) V[:,col]
 * for theta = (l_1..l_d, s, sigma^2): d + 2 doubles.  U_dev, V_dev are n x c
 * (device), alpha_host has c entries.  One pass over all n^2 kernel entries;
 * no kernel block is stored. */
ap_status ap_grad_quadforms(ap_ctx* ctx, const float* U_dev, const float* V_dev, int32_t c,
                            const double* alpha_host, double* out_host);

/* Size of the fixed device scratch array compiled into libap.so for
 * ap_grad_quadforms_static (per GPU that loads the library, held until exit). */
#define AP_STATIC_SCRATCH_BYTES (1u << 20)

/* ap_grad_quadforms without any device allocation.  The paper has no
 * counterpart.  Some callers cannot let a library allocate device memory once
 * their steady state has begun:
 *   - latency-bound serving loops: cudaMalloc and cudaFree synchronise the
 *     whole device, stalling every other stream in flight;
 *   - processes whose own memory pool (an inference server's arena, a
 *     framework's caching allocator) has already reserved the free HBM, so
 *     that a further cudaMalloc fails.
 * Such a caller creates the context once at set-up (ap_create allocates) and
 * then calls this function, which calls no cudaMalloc, no cudaFree and no
 * allocating library routine.
 *   - Same result as ap_grad_quadforms (same kernel; only the order in which
 *     the per-CTA partial sums are added may differ).
 *   - c must be 1, 4, 16 or 32: U_dev and V_dev (n x c, device) are read in
 *     place, without a padding copy.
 *   - Scratch: one AP_STATIC_SCRATCH_BYTES device array shared by every call
 *     in the process, holding (D + 2) doubles per block of 128 rows (256 rows
 *     when D + c <= 40), D = d rounded up to 4, 8, 12, 16, 24 or 32: n up to
 *     about 490k at d = 32 with c = 32 and 3.3M at d <= 8.  A larger problem
 *     returns AP_ERR_SCRATCH_LIMIT before anything is launched.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Work runs on the context's stream (opts.stream); the call copies the
 *     sums to the host and synchronises that stream before it returns.  The
 *     array keeps the last call's contents; each call clears what must start
 *     at zero.  Calls that overlap on the GPU (from several threads or
 *     streams) share the array and race: serialise them. */
ap_status ap_grad_quadforms_static(ap_ctx* ctx, const float* U_dev, const float* V_dev, int32_t c,
                                   const double* alpha_host, double* out_host);

/* Stochastic gradient of the negative MLL (Eq. loss_grad_unbiased): solves
 * K_hat [u, w_1..w_l] = [y - mu, z_1..z_l] with AP, then
 *   g_theta = -1/2 u^T K' u + 1/(2l) sum_i w_i^T K' z_i,  g_mu = -1^T u.
 * y_dev (device, n); Z_dev (device, n x l Rademacher probes) or NULL to draw
 * them from SplitMix64(opts.seed); n_probes = l in [0, 31].
 * grad_host gets d + 3 floats: l_1..l_d, s, sigma^2, mu.  Status as ap_solve. */
ap_status ap_mll_grad(ap_ctx* ctx, const float* y_dev, int32_t n_probes, const float* Z_dev,
                      float* grad_host, ap_info* info);

/* The residual R that Alg. 1 tracked (Eq. text_update_of_r) as the last
 * ap_solve left it: after the last inner step, or after the last FP32
 * recompute when that solve refined or certified (low-precision forms, and
 * the stopping rule).  R_dev (device, n x c) gets it; c must equal the last
 * solve's c.  A verification aid: comparing it with B - K_hat W of the
 * returned W shows the accumulated error of the residual updates.
 * The solve inside ap_mll_grad counts as a solve.  AP_ERR_INVALID_ARG when no
 * solve has left a residual (none yet, a later ap_residual overwrote it, or a
 * call with another padded width resized the buffers) or c differs;
 * AP_ERR_CUDA. */
ap_status ap_tracked_residual(ap_ctx* ctx, int32_t c, float* R_dev);

/* The cudaError_t value of the CUDA call behind this context's last
 * AP_ERR_CUDA (0 if there was none), for diagnostics; 0 for NULL. */
int32_t ap_last_cuda_error(const ap_ctx* ctx);

/* Number of kernels this context has launched since ap_create (all calls). */
int64_t ap_launch_count(const ap_ctx* ctx);

/* Bytes of device memory the context holds right now (scaled inputs, the
 * Cholesky cache, work buffers); 0 for NULL. */
size_t ap_device_bytes(const ap_ctx* ctx);

/* Bounds-checked build only (the library built with AP_CHECKED defined, a
 * separate file from the product library; no counterpart in the paper).
 * Every kernel of that build checks its tile and row indices against the sizes
 * it was given before the accesses they guard; a failing check skips the
 * access and records its source line.  This call synchronises the current
 * device, reads and clears the records of every translation unit, writes
 * "unit:line" of the first one found into where[0..cap) (NUL-terminated, may
 * be NULL) and returns how many units recorded a failure (0: none).  The
 * product build returns -1 and touches nothing. */
int32_t ap_bounds_violations(char* where, int32_t cap);

/* Bounds-checked build only: a one-thread kernel reads element `index` of an
 * 8-element device buffer through the same check, so that an index outside
 * [0, 8) is recorded (and the read skipped) as a failed check; shows that the
 * recording works.  AP_OK, AP_ERR_NOMEM, AP_ERR_CUDA; AP_ERR_UNSUPPORTED in
 * the product build. */
ap_status ap_bounds_selftest(int32_t index);

/* Measured SFU throughput of the current device, in results per SM clock, of
 * the two operations kernel evaluation is made of: ex2.approx (every kernel)
 * and sqrt.approx (Matern kernels).  No counterpart in the paper; the
 * benchmark divides by these rates to place the tensor-core residual update
 * (bound by them) on its roofline.  Runs two probe kernels of about a
 * millisecond on the current device and allocates ~1 MB there while it runs.
 * Both pointers are host doubles.  AP_ERR_INVALID_ARG on NULL, AP_ERR_NOMEM /
 * AP_ERR_CUDA on device errors. */
ap_status ap_sfu_rates(double* ex2_per_clk_sm, double* sqrt_per_clk_sm);

/* The kernel profile phi(r^2) in FP64 exactly as the Cholesky cache evaluates
 * it on the device when it builds the diagonal blocks K_II (Sec. 3, "Cached
 * Cholesky Factors"; phi of Sec. 5: RBF e^{-r^2/2}, Matern-3/2 (1 + u) e^{-u}
 * with u = sqrt(3) r, Matern-5/2 (1 + u + u^2/3) e^{-u} with u = sqrt(5) r),
 * for verification against a host math library.  r2_host and phi_host are
 * host arrays of count doubles (r2 >= 0, finite); the call copies them through
 * device memory it allocates and frees, on the current device, and returns
 * when phi_host is written.  AP_ERR_INVALID_ARG for an unknown kernel, a
 * negative count or NULL arrays with count > 0; AP_ERR_NOMEM / AP_ERR_CUDA on
 * device errors. */
ap_status ap_phi_fp64_eval(int32_t kernel, const double* r2_host, int64_t count, double* phi_host);

/* ------------------------------------------------------------------ serving
 * Continuous batching of GP solve + posterior-mean requests (no counterpart in
 * the paper, which solves one system at a time): requests are admitted in
 * arrival order as soon as a worker slot is free and the request's estimated
 * device footprint fits in the HBM budget; each admitted request runs its own
 * context (cache, Alg. 1 with one CUDA graph per epoch, posterior mean) on its
 * worker's stream, so requests overlap on the device.  Results are
 * deterministic: the same alone and in a mix. */
typedef struct ap_server ap_server;

/* One request.  All host buffers are owned by the caller and must stay valid
 * until the request is done (inputs are copied to the device when the request
 * starts; mean_host is written when it finishes). */
typedef struct ap_request {
    const float* X_host;      /* n x d training inputs */
    int64_t n;
    int32_t d;
    const float* y_host;      /* n labels; the solve is K_hat w = y - hyper.mean */
    const float* Xtest_host;  /* M x d test inputs */
    int64_t M;
    ap_hyper hyper;           /* lengthscales copied at submit */
    int64_t block;
    double tol;
    int32_t stop;             /* ap_stop */
    int32_t min_epochs;
    int32_t max_epochs;
    int32_t precision;        /* ap_precision */
    int32_t refine_every;
    float* mean_host;         /* out: M posterior means */
} ap_request;

typedef struct ap_request_result {
    int32_t done;             /* 1 once finished */
    ap_status status;         /* of the solve (OK, NOT_CONVERGED, ...) once done */
    int32_t epochs;
    double rel_res;           /* ||r||/||y - mu|| reported by the solve */
    double queue_s;           /* submit -> start */
    double latency_s;         /* submit -> result written */
    size_t reserved_bytes;    /* HBM reserved for the request while it runs */
    int32_t started;          /* 1 once a worker has taken the request */
    int32_t compensated;      /* rel_res comes from the compensated recompute */
} ap_request_result;

/* Start a server on device `device` with `slots` worker streams and an HBM
 * budget in bytes.  Errors: INVALID_ARG, CUDA. */
ap_status ap_server_create(ap_server** out, size_t hbm_budget, int32_t slots, int32_t device);
/* Queue a request; *id identifies it.  NOMEM if it can never fit the budget. */
ap_status ap_server_submit(ap_server* srv, const ap_request* req, int64_t* id);
/* Non-blocking status of a request. */
ap_status ap_server_poll(ap_server* srv, int64_t id, ap_request_result* res);
/* Wait up to timeout_s seconds for a request; TIMEOUT if it is not done. */
ap_status ap_server_wait(ap_server* srv, int64_t id, double timeout_s, ap_request_result* res);
/* Cancel a request.  A request not yet started is dropped; a running one
 * stops at the end of its current epoch.  Either way it finishes with status
 * AP_ERR_CANCELLED and writes no posterior mean.  Other requests are not
 * affected.  A request already done keeps its result.  INVALID_ARG for an
 * unknown id. */
ap_status ap_server_cancel(ap_server* srv, int64_t id);
/* Finish admitted requests, drop the rest, stop the workers. */
void ap_server_destroy(ap_server* srv);

/* Release everything the context owns.  NULL is allowed. */
void ap_destroy(ap_ctx* ctx);

/* Static, human-readable name of a status code. */
const char* ap_status_str(ap_status s);

/* Size in bytes of the structs above, for bindings that mirror them. */
size_t ap_sizeof_opts(void);
size_t ap_sizeof_info(void);
size_t ap_sizeof_hyper(void);
size_t ap_sizeof_request(void);
size_t ap_sizeof_request_result(void);

#ifdef __cplusplus
}
#endif
#endif /* AP_H */
