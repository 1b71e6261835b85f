"""Derived error bounds of the tensor-core form of the AP residual update
(Eq. text_update_of_r) and their propagation through Alg. 1, used by the
parity tests in place of measured tolerances.

Entry error.  The tensor-core update evaluates every kernel entry from the
GPU's scaled inputs z = fl32(x * fl32(c_K / l)) * f (f = 1 for RBF, log2(e) for
Matern) and t = |z_i - z_j|^2, with phi = 2^-t (RBF) or, with u = sqrt(t) /
log2(e), (1 + u) e^-u and (1 + u + u^2 / 3) e^-u (Matern-3/2 and -5/2; Sec. 5).
With a_i = |z_i|^2 and u22 = 2^-22 the error of one product term obeys
    |fl(K_ij Delta_j) - K_ij Delta_j| <= w_ij |Delta_j|,
    w_ij = 1.01 s phi_ij (eps_1 + c_K (eps_d (a_i + a_j) + eps_d0)),
where
  * eps_d (a_i + a_j) + eps_d0 bounds the error of t:
      - the two FP32 roundings of the scaled inputs (2^-23 |z| per coordinate)
        move t by at most 2^-21 (a_i + a_j);
      - FP16 hi/lo pairs (hi = fp16(z), lo = fp16(z - hi), plus the FP32 cast
        before the split) carry z to 2^-22 |z| + 2^-25, and dropping lo * lo'
        costs 2^-21 |z_i z_j|: 3.5 u22 (a_i + a_j) + 2^-24 sqrt(d)(|z_i| + |z_j|)
        over the d cross terms;
      - the hi/lo pair of a = |z|^2: 1.25 u22 a;
      - FP32 accumulation inside the tensor cores: at most 2 units of 2^-23
        of (accumulator + |terms|) per MMA of K = 16, n_mma = kdp / 16 MMAs,
        |terms| <= 2 (a_i + a_j): 2 n_mma u22 (a_i + a_j);
    so eps_d = (7 + 2 n_mma) u22 + 2^-25 sqrt(d) (using |z| <= (1 + |z|^2) / 2)
    and eps_d0 = 2^-24 (1 + sqrt(d));
  * c_K bounds |dphi/dt| / phi: ln 2 (RBF), 1 / (2 log2(e)^2) (Matern-3/2),
    1 / (6 log2(e)^2) (Matern-5/2);
  * eps_1 = eps_bf16 + eps_sfu + eps_acc with
      - eps_bf16 = 3 * 2^-18 = 48 u22: phi and Delta as BF16 hi/lo pairs (each
        to 2^-18 relative, the hi parts exact, lo * lo dropped);
      - eps_sfu: ex2.approx and sqrt.approx taken at 4 units of 2^-24
        (2^-21) each; Matern's exponent carries sqrt's error times u, bounded
        for u <= 30 (beyond it phi < 4e-11 and the entry's absolute error is
        below 1e-15 s, the floor abs_floor): RBF 2.25 u22, Matern 67.5 u22;
      - eps_acc = (b / 16 + 2) u22: the FP32 accumulation of the contraction
        over the b / 16 MMAs of a block plus the two partial sums (and the
        boundary slot of a tile shared by two CTAs);
  * 1.01 covers the second-order terms (products of two relative errors,
    |dphi/dt| evaluated over an interval of width |delta t|).
The FP32 epilogue R_i <- R_i - s acc_i (- sigma^2 Delta_i on the index
diagonal) rounds twice: 2^-23 |R_i| per step.

Propagation.  If the GPU's tracked residual after t steps is R_t and its
iterate W_t, the residual lemma (App. B) gives R_t = B - K_hat W_t - e_t with
    |e_t| <= beta_t = sum_{tau < t} w |Delta_tau| + 2^-23 sum_{tau <= t} |R_tau|,
i.e. beta_t = 1.01 s [(eps_1 + c_K eps_d0 + c_K eps_d a) * (K A_t)
                      + c_K eps_d K (a * A_t)] + floor + 2^-23 sum |R_tau|
with A_t = sum_{tau < t} |Delta_tau| (K_hat in place of s phi: the noise
diagonal only adds to the bound).  The FP64 replay of the same block sequence
(W_ref) and the GPU iterate differ by d_t = W_t - W_ref,t with
    d_{t+1} = T_I d_t + P_I (rho_t - K_II^{-1} e_{t,I}),
T_I = I - P_I K_II^{-1} K_hat_{I,:} the K_hat-orthogonal projection of Alg. 1
(norm 1 in the K_hat norm) and rho_t = Delta_t - K_II^{-1} R_{t,I} the block
solve's own rounding (FP32 inverse factor), so
    ||d_k||_K <= sum_t ||beta_{t,I_t}||_2 / sqrt(lambda_min(K_II))
                 + sum_t sqrt(rho_t^T K_II rho_t),
    max_i |d_k,i| <= ||d_k||_K / sqrt(lambda_min(K_hat)) <= ||d_k||_K / sigma.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

U22 = 2.0 ** -22
LOG2E = 1.4426950408889634
RBF, MATERN32, MATERN52 = 0, 1, 2


def scaled_inputs(kernel: int, X: np.ndarray, ell: np.ndarray) -> np.ndarray:
    """The GPU's scaled coordinates z (FP32 products of FP32 scales, times the fold)."""
    ks = {RBF: math.sqrt(0.5 * LOG2E), MATERN32: math.sqrt(3.0), MATERN52: math.sqrt(5.0)}[kernel]
    sh = (ks / np.asarray(ell, dtype=np.float64)).astype(np.float32)
    xs = (np.asarray(X, dtype=np.float32) * sh[None, :]).astype(np.float32)
    fold = 1.0 if kernel == RBF else LOG2E
    return xs.astype(np.float64) * fold


class TcErrorModel:
    """Per-entry bound w_ij of the tensor-core form and its products with |Delta|."""

    def __init__(self, p, kdp: int):
        self.h = oracle.Hyper.of(p)
        self.X = np.asarray(p.X, dtype=np.float64)
        d = p.d
        z = scaled_inputs(p.kernel, p.X, p.lengthscale)
        self.a = (z * z).sum(axis=1)
        n_mma = kdp // 16
        self.eps_d = (7 + 2 * n_mma) * U22 + 2.0 ** -25 * math.sqrt(d)
        self.eps_d0 = 2.0 ** -24 * (1.0 + math.sqrt(d))
        self.c_k = {RBF: math.log(2.0), MATERN32: 1.0 / (2 * LOG2E ** 2), MATERN52: 1.0 / (6 * LOG2E ** 2)}[p.kernel]
        eps_sfu = 2.25 * U22 if p.kernel == RBF else 67.5 * U22
        eps_acc = (p.block / 16 + 2) * U22
        self.eps_1 = 48 * U22 + eps_sfu + eps_acc
        self.floor = 0.0 if p.kernel == RBF else 1e-15 * float(p.outputscale)

    def k_times(self, V: np.ndarray, rows=None) -> np.ndarray:
        """K_hat V (rows of it) by the oracle, V >= 0."""
        return -oracle.residual_rows(self.h, self.X, np.zeros_like(V), V, rows=rows)

    def beta(self, A: np.ndarray, rows=None) -> np.ndarray:
        """Bound on the accumulated update error for accumulated |Delta| sums A
        (n x c), at `rows` (all rows when None); without the R rounding term."""
        a_r = self.a if rows is None else self.a[np.asarray(rows)]
        KA = self.k_times(A, rows)
        KaA = self.k_times(self.a[:, None] * A, rows)
        coef = self.eps_1 + self.c_k * self.eps_d0 + self.c_k * self.eps_d * a_r
        return 1.01 * (coef[:, None] * KA + self.c_k * self.eps_d * KaA) + self.floor * A.sum(axis=0)[None, :]


R_ROUND = 2.0 ** -23  # two FP32 roundings per step of the epilogue's R update
