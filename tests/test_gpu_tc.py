"""Parity of the tensor-core form (AP_BF16_REFINE) with the FP64 oracle, under
tolerances derived from the form's arithmetic (tests/error_model.py):

  * every step of a 2m + 1 step run: the GPU's Gauss-Southwell choice is the
    argmax of its own tracked block norms, and on the chosen block's rows the
    tracked residual equals B - K_hat W of the GPU's iterate up to the derived
    bound beta_t of the accumulated update error (Eq. text_update_of_r and the
    residual lemma of App. B);
  * after the run, the same holds on every row, and the FP64 oracle's replay
    of the GPU's block sequence (Alg. 1 with forced choices) differs from the
    GPU's W by no more than the propagated bound, in the K_hat norm and
    element by element.

The GPU's per-step iterates come from one run per step count (max_steps = t):
the runs are deterministic, and each repeats the block sequence of the longest
one (checked).  Accuracy of whole solves is won back by the FP32 residual
recompute (refinement), tested last.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2310_17137_gb300 as ap
import workloads as wl
from error_model import R_ROUND, TcErrorModel

pytestmark = pytest.mark.gpu

CASES = [
    # n, d, b, c, kernel: several 128-row tiles and 128-column chunks, ragged
    # tails; distance operands of K = 16, 32, 64, 48 and 96 (3d + 4 rounded up
    # to 16; d = 30 is the largest the tensor-core form takes, with the largest
    # shared-memory stages at c = 32)
    (1000, 3, 256, 16, wl.MATERN52),
    (1337, 5, 300, 3, wl.RBF),
    (777, 17, 192, 32, wl.MATERN32),
    (2100, 11, 512, 16, wl.RBF),
    (900, 30, 384, 32, wl.MATERN52),
    # more 128-row tiles (162) than SMs, so the work ranges of the persistent
    # CTAs split tiles between two CTAs (boundary slots)
    (20600, 3, 256, 16, wl.MATERN52),
    (20600, 5, 384, 32, wl.RBF),
]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def tc_kd(d):
    return (3 * d + 4 + 15) // 16 * 16


def _ctx(p, X=None, trace_cap=0, **kw):
    opts = ap.ap_opts_default(block=p.block, precision=ap.AP_BF16_REFINE, **kw)
    return ap.ap_create(_t(p.X) if X is None else X, ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise,
                                                              p.mean), opts, trace_cap=trace_cap)


def _gpu_after(p, X, B, t):
    """(W, tracked R, block trace) of the GPU after exactly t steps."""
    ctx = _ctx(p, X, trace_cap=max(t, 1), tol=1e-30, min_epochs=0, max_steps=t, refine_every=0)
    st, W, info, trace = ap.ap_solve(ctx, B)
    assert st == ap.AP_ERR_NOT_CONVERGED and info["steps"] == t
    R = ap.ap_tracked_residual(ctx, p.c)
    out = _f64(W.cpu().numpy()), _f64(R.cpu().numpy()), np.asarray(trace[:t])
    ap.ap_destroy(ctx)
    return out


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}d{c[1]}b{c[2]}c{c[3]}k{c[4]}")
def test_tc_steps_within_derived_bounds(case):
    n, d, b, c, kern = case
    p = wl.random_problem(n, d, b, c, kern, 0.05, 21)
    m = -(-n // b)
    k = 2 * m + 1
    em = TcErrorModel(p, tc_kd(d))
    h, X, B = em.h, em.X, _f64(p.B)
    Xd, Bd = _t(p.X), _t(p.B)
    W_k, R_k, trace = _gpu_after(p, Xd, Bd, k)
    blocks = {}

    def block(J):
        if J not in blocks:
            lo, hi = J * b, min(n, J * b + b)
            K = oracle.gram(h, X[lo:hi], X[lo:hi], row0=lo, col0=lo)
            blocks[J] = (np.arange(lo, hi), K, oracle.cholesky(K), np.linalg.eigvalsh(K)[0])
        return blocks[J]

    A = np.zeros((n, c))      # sum of |Delta_tau| so far
    SR = np.abs(B)            # sum of |R_tau| so far (R_0 = B)
    S_K = np.zeros(c)         # propagated bound on ||W_gpu - W_ref||_K, per column
    W_t, R_t = np.zeros((n, c)), B.copy()
    worst_e = 0.0
    for t in range(k):
        I = int(trace[t])
        rows, K_II, L_II, lam = block(I)
        # Gauss-Southwell: the GPU chose the largest block norm of its own residual
        norms = np.array([np.sum(R_t[J * b:min(n, J * b + b)] ** 2) for J in range(m)])
        assert norms[I] >= norms.max() * (1 - 1e-5), (t, I, norms.argmax())
        # update error accumulated on the chosen rows
        beta_I = em.beta(A, rows) + R_ROUND * SR[rows]
        e_I = oracle.residual_rows(h, X, B, W_t, rows=rows) - R_t[rows]
        assert np.all(np.abs(e_I) <= beta_I), (t, np.max(np.abs(e_I) / beta_I))
        worst_e = max(worst_e, float(np.max(np.abs(e_I) / beta_I)))
        # the next iterate; its block-solve rounding against K_II^{-1} R_I
        W_n, R_n, tr = _gpu_after(p, Xd, Bd, t + 1) if t + 1 < k else (W_k, R_k, trace)
        np.testing.assert_array_equal(tr, trace[:t + 1])
        delta = W_n[rows] - W_t[rows]
        rho = delta - oracle.chol_solve(L_II, R_t[rows])
        S_K += np.linalg.norm(beta_I, axis=0) / np.sqrt(lam) + np.sqrt(np.einsum("ic,ij,jc->c", rho, K_II, rho))
        A[rows] += np.abs(delta)
        W_t, R_t = W_n, R_n
        SR += np.abs(R_t)
    # every row after the last step
    beta = em.beta(A) + R_ROUND * SR
    e = oracle.residual_rows(h, X, B, W_k) - R_k
    assert np.all(np.abs(e) <= beta), np.max(np.abs(e) / beta)
    # the FP64 replay of the same block sequence
    r = oracle.ap_solve(h, X, B, b, select=oracle.SEL_FORCED, forced=trace, max_steps=k, trace_cap=k)
    np.testing.assert_array_equal(r.trace, trace)
    dW = W_k - r.W
    dK = np.sqrt(np.maximum(np.sum(dW * em.k_times(dW), axis=0), 0.0))
    assert np.all(dK <= S_K), dK / S_K
    assert np.all(np.abs(dW).max(axis=0) <= S_K / np.sqrt(p.noise)), np.abs(dW).max(axis=0) * np.sqrt(p.noise) / S_K
    print(f"{case}: update error / bound {max(worst_e, float(np.max(np.abs(e) / beta))):.3f}, "
          f"||dW||_K / bound {float(np.max(dK / S_K)):.3f}, max|dW| / max|W| {np.abs(dW).max() / np.abs(r.W).max():.2e}")


def test_tc_solve_with_refinement_reaches_fp32_accuracy():
    p = wl.random_problem(3000, 5, 256, 16, wl.MATERN52, 0.1, 23, ell_range=(0.1, 0.3))
    ctx = _ctx(p, tol=1e-5, stop=ap.AP_STOP_MAX_REL, min_epochs=1, max_epochs=500, refine_every=3)
    st, W, info, _ = ap.ap_solve(ctx, _t(p.B))
    assert st == ap.AP_OK, info
    assert info["refinements"] >= 1
    R = oracle.residual_rows(oracle.Hyper.of(p), _f64(p.X), _f64(p.B), _f64(W.cpu().numpy()))
    rel = np.linalg.norm(R, axis=0) / np.linalg.norm(p.B, axis=0)
    assert rel.max() <= 1.2e-5, rel
