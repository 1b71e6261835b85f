/*
 * FP64 CPU oracle for the alternating-projection (AP) GP solver.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path and includes nothing from
 * it.  Everything is plain, slow, double precision, written from the paper:
 *
 *   Wu, Wenger, Bindel, Gardner, Pleiss, Cunningham, Gardner:
 *   "Large-Scale Gaussian Processes via Alternating Projection", AISTATS 2024.
 *
 * Two independent parts:
 *   (1) the definition: dense kernel matrix, own Cholesky, exact solve,
 *       posterior mean, exact MLL and its gradient (Sec. 2, Eq. loss and
 *       Eq. loss_grad_unbiased);
 *   (2) the algorithm: Alg. 1 (alternating projection) step by step with the
 *       modified Gauss-Southwell rule (Eq. approximate_gauss_southwell), the
 *       cached block Cholesky factors (Sec. 3, "Cached Cholesky Factors"), the
 *       sequential partition and the stopping rule of Sec. 5; and Alg. 2
 *       (block coordinate descent, App. B) as a second formulation.
 *
 * Readings of the paper used here (the paper is silent on them):
 *   - kernel k(x,x') = s * phi(r), r = ||(x - x') / lengthscale||, with
 *     RBF phi = exp(-r^2/2), Matern-3/2 phi = (1 + sqrt3 r) exp(-sqrt3 r),
 *     Matern-5/2 phi = (1 + sqrt5 r + 5 r^2 / 3) exp(-sqrt5 r);
 *   - the noise sigma^2 sits on the index diagonal (Sec. 2 footnote read as
 *     sigma^2 I), so K_hat = s phi + sigma^2 I and K(X*, X) has no noise;
 *   - Gauss-Southwell ties go to the smallest block index;
 *   - the residual update of Alg. 1 runs over all n rows, rows of I included.
 *
 * Layouts: all matrices row-major.  X is n x d, B/W/R are n x c.
 * OpenMP runs independent rows (or columns) in parallel; it never changes the
 * order of any sum.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_RBF = 0, ORC_MATERN32 = 1, ORC_MATERN52 = 2 };
enum { ORC_SEL_GS = 0, ORC_SEL_CYCLIC = 1, ORC_SEL_FORCED = 2 };
enum { ORC_STOP_MEAN_REL = 0, ORC_STOP_MAX_REL = 1, ORC_STOP_FRO = 2, ORC_STOP_Y_REL = 3 };
enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_NOT_SPD = 2, ORC_BAD_ARG = 3 };

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- kernels */

/* Squared scaled distance sum_k ((x_k - x'_k) / l_k)^2 by direct differences. */
static double scaled_r2(int d, const double* ell, const double* xi, const double* xj) {
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = (xi[k] - xj[k]) / ell[k];
        r2 += t * t;
    }
    return r2;
}

/* phi(r) as a function of r^2 (Rasmussen & Williams ch. 4 forms). */
static double phi_of_r2(int kind, double r2) {
    if (kind == ORC_RBF) return exp(-0.5 * r2);
    if (kind == ORC_MATERN32) {
        double u = sqrt(3.0 * r2);
        return (1.0 + u) * exp(-u);
    }
    double u = sqrt(5.0 * r2);
    return (1.0 + u + u * u / 3.0) * exp(-u);
}

/* d phi / d (r^2), written without a division by r. */
static double dphi_dr2(int kind, double r2) {
    if (kind == ORC_RBF) return -0.5 * exp(-0.5 * r2);
    if (kind == ORC_MATERN32) {
        double u = sqrt(3.0 * r2);
        return -1.5 * exp(-u);
    }
    double u = sqrt(5.0 * r2);
    return -(5.0 / 6.0) * (1.0 + u) * exp(-u);
}

double orc_kernel_value(int kind, int d, const double* ell, double s,
                        const double* xi, const double* xj) {
    return s * phi_of_r2(kind, scaled_r2(d, ell, xi, xj));
}

/* Dense block of K_hat: out[i][j] = s phi(x_a[i], x_b[j]) + noise [row0+i == col0+j].
 * row0/col0 are the global indices of the first row/column; pass noise = 0
 * for cross-covariances with test points. */
void orc_gram(int kind, int d, const double* ell, double s, double noise,
              const double* Xa, int64_t na, int64_t row0,
              const double* Xb, int64_t nb, int64_t col0, double* out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < na; ++i)
        for (int64_t j = 0; j < nb; ++j) {
            double v = orc_kernel_value(kind, d, ell, s, Xa + i * d, Xb + j * d);
            if (row0 + i == col0 + j) v += noise;
            out[i * nb + j] = v;
        }
}

/* ------------------------------------------------------- dense linear algebra */

/* In-place Cholesky A = L L^T (Cholesky-Crout order), lower triangle of the
 * row-major n x n matrix A is overwritten by L and the strict upper triangle
 * is zeroed.  Returns -1 on success, else the index of the first pivot that is
 * not positive. */
int64_t orc_cholesky(int64_t n, double* A) {
    for (int64_t j = 0; j < n; ++j) {
        double djj = A[j * n + j];
        for (int64_t k = 0; k < j; ++k) djj -= A[j * n + k] * A[j * n + k];
        if (!(djj > 0.0)) return j;
        double ljj = sqrt(djj);
        A[j * n + j] = ljj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            double v = A[i * n + j];
            for (int64_t k = 0; k < j; ++k) v -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = v / ljj;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) A[i * n + j] = 0.0;
    return -1;
}

/* Solve L L^T X = B for the c columns of the row-major n x c matrix B. */
void orc_chol_solve(int64_t n, const double* L, int c, const double* B, double* Xout) {
#pragma omp parallel for schedule(static)
    for (int col = 0; col < c; ++col) {
        double* y = (double*)malloc(sizeof(double) * (size_t)n);
        for (int64_t i = 0; i < n; ++i) { /* forward: L y = b */
            double v = B[i * c + col];
            for (int64_t k = 0; k < i; ++k) v -= L[i * n + k] * y[k];
            y[i] = v / L[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) { /* backward: L^T x = y */
            double v = y[i];
            for (int64_t k = i + 1; k < n; ++k) v -= L[k * n + i] * y[k];
            y[i] = v / L[i * n + i];
        }
        for (int64_t i = 0; i < n; ++i) Xout[i * c + col] = y[i];
        free(y);
    }
}

/* Dense exact solve K_hat W = B via the own Cholesky.  Returns -1 or the bad pivot. */
int64_t orc_dense_solve(int kind, int d, const double* ell, double s, double noise,
                        int64_t n, const double* X, int c, const double* B, double* W) {
    double* K = (double*)malloc(sizeof(double) * (size_t)(n * n));
    orc_gram(kind, d, ell, s, noise, X, n, 0, X, n, 0, K);
    int64_t bad = orc_cholesky(n, K);
    if (bad < 0) orc_chol_solve(n, K, c, B, W);
    free(K);
    return bad;
}

/* ------------------------------------------------------------- AP building blocks */

/* Block norms ||R_{J,:}||_F^2 for the sequential partition of block size b, and
 * the Gauss-Southwell choice argmax_J (ties to the smallest J).  Eq.
 * approximate_gauss_southwell. */
int orc_gs_select(int64_t n, int64_t b, int c, const double* R, double* norms_out) {
    int64_t m = (n + b - 1) / b;
    int best = 0;
    double bestv = -1.0;
    for (int64_t J = 0; J < m; ++J) {
        int64_t lo = J * b, hi = lo + b < n ? lo + b : n;
        double acc = 0.0;
        for (int64_t i = lo; i < hi; ++i)
            for (int col = 0; col < c; ++col) acc += R[i * c + col] * R[i * c + col];
        if (norms_out) norms_out[J] = acc;
        if (acc > bestv) { bestv = acc; best = (int)J; }
    }
    return best;
}

/* rows[i] of R -= K_hat(X_rows, X_I) Delta for the given rows: the residual
 * update of Eq. text_update_of_r, kernel entries evaluated one by one.
 * rows == NULL means rows 0..nrows-1. */
void orc_block_update(int kind, int d, const double* ell, double s, double noise,
                      const double* X, int64_t i0, int64_t bI, int c, const double* Delta,
                      int64_t nrows, const int64_t* rows, double* R) {
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows ? rows[t] : t;
        for (int64_t jj = 0; jj < bI; ++jj) {
            int64_t j = i0 + jj;
            double kij = orc_kernel_value(kind, d, ell, s, X + i * d, X + j * d);
            if (i == j) kij += noise;
            for (int col = 0; col < c; ++col) R[i * c + col] -= kij * Delta[jj * c + col];
        }
    }
}

/* Per-column relative residuals ||r_col|| / ||b_col||. */
static void column_rel(int64_t n, int c, const double* R, const double* B, double* rel,
                       double* fro_r, double* fro_b) {
    double fr = 0.0, fb = 0.0;
    for (int col = 0; col < c; ++col) {
        double nr = 0.0, nb = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            nr += R[i * c + col] * R[i * c + col];
            nb += B[i * c + col] * B[i * c + col];
        }
        fr += nr;
        fb += nb;
        rel[col] = nb > 0.0 ? sqrt(nr) / sqrt(nb) : sqrt(nr);
    }
    *fro_r = sqrt(fr);
    *fro_b = sqrt(fb);
}

/* Stopping rules: MEAN_REL is Sec. 5's (average relative residual strictly
 * below tol), FRO is Alg. 1's ||R|| <= tol ||B||, MAX_REL asks every column,
 * Y_REL asks the first (label) column only. */
static int stop_met(int rule, double tol, int c, const double* rel, double fro_r, double fro_b) {
    if (rule == ORC_STOP_FRO) return fro_r <= tol * fro_b;
    if (rule == ORC_STOP_Y_REL) return rel[0] <= tol;
    if (rule == ORC_STOP_MAX_REL) {
        for (int col = 0; col < c; ++col) if (!(rel[col] <= tol)) return 0;
        return 1;
    }
    double mean = 0.0;
    for (int col = 0; col < c; ++col) mean += rel[col];
    return mean / c < tol;
}

/* Energy h(W) = 1/2 tr(W^T K W) - tr(B^T W) evaluated through K W = B - R,
 * i.e. h = -1/2 tr(W^T (B + R)) (App. B, Eq. quadratic-objective with the
 * residual lemma). */
static double energy_via_residual(int64_t n, int c, const double* W, const double* B,
                                  const double* R) {
    double acc = 0.0;
    for (int64_t i = 0; i < n * c; ++i) acc += W[i] * (B[i] + R[i]);
    return -0.5 * acc;
}

/*
 * Alg. 1, alternating projection, in the paper's order:
 *   partition [n] sequentially into m = ceil(n/b) blocks (last one short);
 *   factor every K_hat_{I,I} once (cached Cholesky factors, Sec. 3);
 *   W = 0, R = B;
 *   per epoch, m times: select I; Delta = K_II^{-1} R_I; W_I += Delta;
 *                        R -= K_hat_{:,I} Delta (all n rows);
 *   after each epoch: stop if the rule holds and epoch >= min_epochs, or at
 *   max_epochs.  max_steps > 0 also ends the run after that many steps.
 *
 * select: GS (Eq. approximate_gauss_southwell), CYCLIC (step j picks block
 * j mod m) or FORCED (the caller's sequence, used for random selection with
 * caller-drawn indices and for replaying another implementation's choices).
 *
 * Per-step records (first trace_cap steps, any pointer may be NULL):
 *   trace[j]       chosen block
 *   energy[j]      h(W) after the step
 *   pred_dec[j]    -1/2 tr(R_I^T Delta), the exact change of h (App. C proof)
 *   chosen_norm[j] ||R_I||_F^2 of the chosen block before the step
 *   max_norm[j]    max_J ||R_J||_F^2 before the step
 * Returns ORC_OK, ORC_NOT_CONVERGED or ORC_NOT_SPD (block index in *bad_block).
 */
int orc_ap_solve(int kind, int d, const double* ell, double s, double noise,
                 int64_t n, const double* X, int64_t b, int c, const double* B,
                 int select, const int* forced, int64_t n_forced,
                 int stop_rule, double tol, int min_epochs, int max_epochs, int64_t max_steps,
                 double* W, double* R,
                 int* trace, double* energy, double* pred_dec, double* chosen_norm,
                 double* max_norm, int64_t trace_cap,
                 int64_t* steps_out, int* epochs_out, double* rel_out, int* bad_block) {
    if (n <= 0 || b <= 0 || c <= 0 || d <= 0) return ORC_BAD_ARG;
    int64_t m = (n + b - 1) / b;
    /* cached Cholesky factors of every diagonal block */
    double** Lc = (double**)calloc((size_t)m, sizeof(double*));
    int status = ORC_OK;
    for (int64_t J = 0; J < m; ++J) {
        int64_t lo = J * b, bJ = (lo + b < n ? b : n - lo);
        Lc[J] = (double*)malloc(sizeof(double) * (size_t)(bJ * bJ));
        orc_gram(kind, d, ell, s, noise, X + lo * d, bJ, lo, X + lo * d, bJ, lo, Lc[J]);
        if (orc_cholesky(bJ, Lc[J]) >= 0) {
            if (bad_block) *bad_block = (int)J;
            status = ORC_NOT_SPD;
            break;
        }
    }
    int64_t steps = 0;
    int epoch = 0;
    double* norms = (double*)malloc(sizeof(double) * (size_t)m);
    double* Delta = (double*)malloc(sizeof(double) * (size_t)(b * c));
    double* rel = (double*)malloc(sizeof(double) * (size_t)c);
    if (status == ORC_OK) {
        memset(W, 0, sizeof(double) * (size_t)(n * c));
        memcpy(R, B, sizeof(double) * (size_t)(n * c));
        status = ORC_NOT_CONVERGED;
        int done = 0;
        for (epoch = 1; epoch <= max_epochs && !done; ++epoch) {
            for (int64_t j = 0; j < m; ++j) {
                if (max_steps > 0 && steps >= max_steps) { done = 1; break; }
                int gs = orc_gs_select(n, b, c, R, norms);
                int I;
                if (select == ORC_SEL_CYCLIC) I = (int)(steps % m);
                else if (select == ORC_SEL_FORCED) I = (steps < n_forced) ? forced[steps] : gs;
                else I = gs;
                if (I < 0 || I >= m) { status = ORC_BAD_ARG; done = 1; break; }
                int64_t lo = (int64_t)I * b, bI = (lo + b < n ? b : n - lo);
                orc_chol_solve(bI, Lc[I], c, R + lo * c, Delta);
                double dec = 0.0;
                for (int64_t t = 0; t < bI * c; ++t) dec += R[lo * c + t] * Delta[t];
                for (int64_t t = 0; t < bI * c; ++t) W[lo * c + t] += Delta[t];
                orc_block_update(kind, d, ell, s, noise, X, lo, bI, c, Delta, n, NULL, R);
                if (steps < trace_cap) {
                    if (trace) trace[steps] = I;
                    if (pred_dec) pred_dec[steps] = -0.5 * dec;
                    if (chosen_norm) chosen_norm[steps] = norms[I];
                    if (max_norm) max_norm[steps] = norms[gs];
                    if (energy) energy[steps] = energy_via_residual(n, c, W, B, R);
                }
                ++steps;
            }
            double fr, fb;
            column_rel(n, c, R, B, rel, &fr, &fb);
            if (!done && stop_met(stop_rule, tol, c, rel, fr, fb) && epoch >= min_epochs) {
                status = ORC_OK;
                done = 1;
            }
            if (done) break;
        }
        if (epoch > max_epochs) epoch = max_epochs;
        if (rel_out) {
            double fr, fb;
            column_rel(n, c, R, B, rel, &fr, &fb);
            memcpy(rel_out, rel, sizeof(double) * (size_t)c);
        }
    }
    if (steps_out) *steps_out = steps;
    if (epochs_out) *epochs_out = epoch;
    for (int64_t J = 0; J < m; ++J) free(Lc[J]);
    free(Lc);
    free(norms);
    free(Delta);
    free(rel);
    return status;
}

/*
 * Alg. 2, block coordinate descent, on the block sequence seq[0..steps):
 *   W_I = K_II^{-1} (B_I - K_{I, not I} W_{not I}).
 * It keeps no residual; the off-block products are evaluated from W each step.
 */
int orc_bcd(int kind, int d, const double* ell, double s, double noise,
            int64_t n, const double* X, int64_t b, int c, const double* B,
            const int* seq, int64_t steps, double* W) {
    int64_t m = (n + b - 1) / b;
    memset(W, 0, sizeof(double) * (size_t)(n * c));
    double* rhs = (double*)malloc(sizeof(double) * (size_t)(b * c));
    double* L = (double*)malloc(sizeof(double) * (size_t)(b * b));
    int status = ORC_OK;
    for (int64_t t = 0; t < steps; ++t) {
        int I = seq[t];
        if (I < 0 || I >= m) { status = ORC_BAD_ARG; break; }
        int64_t lo = (int64_t)I * b, bI = (lo + b < n ? b : n - lo);
#pragma omp parallel for schedule(static)
        for (int64_t ii = 0; ii < bI; ++ii) {
            int64_t i = lo + ii;
            for (int col = 0; col < c; ++col) {
                double v = B[i * c + col];
                for (int64_t j = 0; j < n; ++j) {
                    if (j >= lo && j < lo + bI) continue;
                    v -= orc_kernel_value(kind, d, ell, s, X + i * d, X + j * d) * W[j * c + col];
                }
                rhs[ii * c + col] = v;
            }
        }
        orc_gram(kind, d, ell, s, noise, X + lo * d, bI, lo, X + lo * d, bI, lo, L);
        if (orc_cholesky(bI, L) >= 0) { status = ORC_NOT_SPD; break; }
        orc_chol_solve(bI, L, c, rhs, W + lo * c);
    }
    free(rhs);
    free(L);
    return status;
}

/* True residual rows r_i = b_i - sum_j K_hat_ij w_j for the requested rows
 * (rows == NULL: rows 0..nrows-1).  out is nrows x c. */
void orc_residual_rows(int kind, int d, const double* ell, double s, double noise,
                       int64_t n, const double* X, int c, const double* B, const double* W,
                       int64_t nrows, const int64_t* rows, double* out) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows ? rows[t] : t;
        for (int col = 0; col < c; ++col) out[t * c + col] = B[i * c + col];
        for (int64_t j = 0; j < n; ++j) {
            double kij = orc_kernel_value(kind, d, ell, s, X + i * d, X + j * d);
            if (i == j) kij += noise;
            for (int col = 0; col < c; ++col) out[t * c + col] -= kij * W[j * c + col];
        }
    }
}

/* Posterior mean mu + K(X*, X) w (Sec. 2): no noise term on the cross kernel. */
void orc_predict_mean(int kind, int d, const double* ell, double s, double mean,
                      int64_t n, const double* X, const double* w,
                      int64_t M, const double* Xs, double* out) {
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < M; ++t) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j)
            acc += orc_kernel_value(kind, d, ell, s, Xs + t * d, X + j * d) * w[j];
        out[t] = mean + acc;
    }
}

/* dK_hat_ij / dtheta for theta = (l_1..l_d, s, sigma^2); index p in [0, d+2). */
static double dkhat(int kind, int d, const double* ell, double s, int64_t i, int64_t j,
                    const double* xi, const double* xj, int p) {
    if (p == d + 1) return i == j ? 1.0 : 0.0;
    double r2 = scaled_r2(d, ell, xi, xj);
    if (p == d) return phi_of_r2(kind, r2);
    double diff = xi[p] - xj[p];
    /* dr2/dl_p = -2 diff^2 / l_p^3 */
    return s * dphi_dr2(kind, r2) * (-2.0 * diff * diff / (ell[p] * ell[p] * ell[p]));
}

/*
 * Quadratic forms g_p = sum_col alpha[col] U[:,col]^T (dK_hat/dtheta_p) V[:,col]
 * for p over (l_1..l_d, s, sigma^2): the building block of Eq.
 * loss_grad_unbiased.  U, V are n x c.  out has d + 2 entries.
 */
void orc_grad_quadforms(int kind, int d, const double* ell, double s,
                        int64_t n, const double* X, int c, const double* U, const double* V,
                        const double* alpha, double* out) {
    int P = d + 2;
    for (int p = 0; p < P; ++p) out[p] = 0.0;
#pragma omp parallel
    {
        double* loc = (double*)calloc((size_t)P, sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                double g = 0.0;
                for (int col = 0; col < c; ++col) g += alpha[col] * U[i * c + col] * V[j * c + col];
                for (int p = 0; p < P; ++p)
                    loc[p] += g * dkhat(kind, d, ell, s, i, j, X + i * d, X + j * d, p);
            }
        }
#pragma omp critical
        for (int p = 0; p < P; ++p) out[p] += loc[p];
        free(loc);
    }
}

/*
 * Exact negative MLL (Eq. loss without the n/2 log 2pi constant)
 *   l = 1/2 ((y - mu)^T K_hat^{-1} (y - mu) + log det K_hat)
 * and its exact gradient
 *   dl/dtheta = -1/2 u^T K' u + 1/2 tr(K_hat^{-1} K'),  u = K_hat^{-1}(y - mu),
 *   dl/dmu    = -1^T u,
 * for theta = (l_1..l_d, s, sigma^2, mu): grad has d + 3 entries.
 * Dense, O(n^3).  Returns -1 or the bad pivot.
 */
int64_t orc_mll_exact(int kind, int d, const double* ell, double s, double noise, double mean,
                      int64_t n, const double* X, const double* y, double* mll, double* grad) {
    double* L = (double*)malloc(sizeof(double) * (size_t)(n * n));
    orc_gram(kind, d, ell, s, noise, X, n, 0, X, n, 0, L);
    int64_t bad = orc_cholesky(n, L);
    if (bad >= 0) { free(L); return bad; }
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* u = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) r[i] = y[i] - mean;
    orc_chol_solve(n, L, 1, r, u);
    double quad = 0.0, logdet = 0.0;
    for (int64_t i = 0; i < n; ++i) quad += r[i] * u[i];
    for (int64_t i = 0; i < n; ++i) logdet += 2.0 * log(L[i * n + i]);
    *mll = 0.5 * (quad + logdet);
    if (grad) {
        /* K_hat^{-1} column by column from the factor */
        double* Kinv = (double*)malloc(sizeof(double) * (size_t)(n * n));
        double* Id = (double*)calloc((size_t)(n * n), sizeof(double));
        for (int64_t i = 0; i < n; ++i) Id[i * n + i] = 1.0;
        orc_chol_solve(n, L, (int)n, Id, Kinv);
        free(Id);
        int P = d + 2;
        for (int p = 0; p < P; ++p) grad[p] = 0.0;
#pragma omp parallel
        {
            double* loc = (double*)calloc((size_t)P, sizeof(double));
#pragma omp for schedule(static)
            for (int64_t i = 0; i < n; ++i)
                for (int64_t j = 0; j < n; ++j)
                    for (int p = 0; p < P; ++p) {
                        double dk = dkhat(kind, d, ell, s, i, j, X + i * d, X + j * d, p);
                        loc[p] += -0.5 * u[i] * dk * u[j] + 0.5 * Kinv[i * n + j] * dk;
                    }
#pragma omp critical
            for (int p = 0; p < P; ++p) grad[p] += loc[p];
            free(loc);
        }
        double gmu = 0.0;
        for (int64_t i = 0; i < n; ++i) gmu -= u[i];
        grad[d + 2] = gmu;
        free(Kinv);
    }
    free(L);
    free(r);
    free(u);
    return -1;
}

/*
 * The stochastic estimator of Eq. loss_grad_unbiased with the caller's probes
 * Z (n x l), every solve done exactly (dense):
 *   g = -1/2 u^T K' u + 1/(2l) sum_i (K_hat^{-1} z_i)^T K' z_i,  dl/dmu = -1^T u.
 * grad has d + 3 entries.  Returns -1 or the bad pivot.
 */
int64_t orc_mll_grad_stochastic(int kind, int d, const double* ell, double s, double noise,
                                double mean, int64_t n, const double* X, const double* y,
                                int l, const double* Z, double* grad) {
    int c = l + 1;
    double* Bm = (double*)malloc(sizeof(double) * (size_t)(n * c));
    double* Wm = (double*)malloc(sizeof(double) * (size_t)(n * c));
    for (int64_t i = 0; i < n; ++i) {
        Bm[i * c] = y[i] - mean;
        for (int k = 0; k < l; ++k) Bm[i * c + 1 + k] = Z[i * l + k];
    }
    int64_t bad = orc_dense_solve(kind, d, ell, s, noise, n, X, c, Bm, Wm);
    if (bad >= 0) { free(Bm); free(Wm); return bad; }
    /* U = [u, w_1..w_l], V = [u, z_1..z_l], alpha = [-1/2, 1/(2l), ...] */
    double* alpha = (double*)malloc(sizeof(double) * (size_t)c);
    double* V = (double*)malloc(sizeof(double) * (size_t)(n * c));
    alpha[0] = -0.5;
    for (int k = 0; k < l; ++k) alpha[1 + k] = 0.5 / l;
    for (int64_t i = 0; i < n; ++i) {
        V[i * c] = Wm[i * c];
        for (int k = 0; k < l; ++k) V[i * c + 1 + k] = Z[i * l + k];
    }
    orc_grad_quadforms(kind, d, ell, s, n, X, c, Wm, V, alpha, grad);
    double gmu = 0.0;
    for (int64_t i = 0; i < n; ++i) gmu -= Wm[i * c];
    grad[d + 2] = gmu;
    free(Bm);
    free(Wm);
    free(alpha);
    free(V);
    return -1;
}
