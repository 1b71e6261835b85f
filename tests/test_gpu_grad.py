"""The MLL gradient at the check size of the gradient workload: n = 4096,
d = 8, Matern-3/2 ARD, noise 0.05, 31 Rademacher probes, 8 blocks of 512
(Eq. loss_grad_unbiased, Sec. 2), through ap_mll_grad, against the FP64 oracle.

Every derivative matrix dK_hat/dtheta of this family has non-negative entries
(phi decreases in r, and r^2 decreases in every lengthscale; dK/ds = phi;
dK_hat/dsigma^2 = I), so |a^T K' b| <= |a|^T K' |b| and the oracle's quadratic
forms on absolute values bound every error term:

  * kernel arithmetic: on the GPU's own solution W (the same deterministic solve
    through ap_solve), |g_gpu - g(W)| <= 1e-5 |W|^T K' |V|, the FP32 product
    tolerance of the quadratic-form kernel;
  * solve error: with E = W - W* (W* the dense FP64 solve), the data-fit term
    changes by at most |E_0|^T K' (|W*_0| + |E_0| / 2) and each probe term by
    |E_i|^T K' |z_i| / (2l); the mean component by sum |E_0|.
So the GPU gradient must lie within their sum of the oracle's estimator with
the same probes and exact solves, element by element.  The distance to the
exact gradient (dense trace) is the estimator's own noise and is reported.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2310_17137_gb300 as ap
import workloads as wl

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")


def test_mll_grad_n4096_matern32_31_probes_against_oracle():
    p = wl.matern32_grad(n=4096, block=512)
    l = p.c - 1
    Z = np.ascontiguousarray(p.B[:, 1:])
    h = oracle.Hyper.of(p)
    X64, B64, Z64 = p.X.astype(np.float64), p.B.astype(np.float64), Z.astype(np.float64)
    tol = 1e-4
    opts = ap.ap_opts_default(block=p.block, tol=tol, stop=ap.AP_STOP_MAX_REL, min_epochs=1, max_epochs=50000)
    ctx = ap.ap_create(_t(p.X), ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean), opts)
    st, g, info = ap.ap_mll_grad(ctx, _t(p.y), l, _t(Z))
    assert st == ap.AP_OK, info
    # the same solve through ap_solve: the GPU's own W
    st2, W, info2, _ = ap.ap_solve(ctx, _t(p.B))
    assert st2 == ap.AP_OK and info2["epochs"] == info["epochs"]
    W = W.cpu().numpy().astype(np.float64)
    # every column certified by the oracle's FP64 residual
    R = oracle.residual_rows(h, X64, B64, W)
    rel = np.linalg.norm(R, axis=0) / np.linalg.norm(B64, axis=0)
    assert rel.max() <= 1.05 * tol, rel
    d = p.d
    alpha = np.array([-0.5] + [0.5 / l] * l)
    V = np.concatenate([W[:, :1], Z64], axis=1)
    # kernel arithmetic on the GPU's own solution
    q_own = oracle.grad_quadforms(h, X64, W, V, alpha)
    mag = oracle.grad_quadforms(h, X64, np.abs(W), np.abs(V), np.abs(alpha))
    g = np.asarray(g, dtype=np.float64)
    tol_kernel = 1e-5 * mag + 2.0 ** -23 * np.abs(q_own)
    assert np.all(np.abs(g[:d + 2] - q_own) <= tol_kernel), (g[:d + 2], q_own)
    # solve error, bounded with the non-negative derivative matrices
    Wstar = oracle.dense_solve(h, X64, B64)
    E = np.abs(W - Wstar)
    U = E
    Vb = np.concatenate([np.abs(Wstar[:, :1]) + 0.5 * E[:, :1], np.abs(Z64)], axis=1)
    ab = np.array([1.0] + [0.5 / l] * l)
    tol_solve = oracle.grad_quadforms(h, X64, U, Vb, ab)
    ref = oracle.mll_grad_stochastic(h, X64, p.y.astype(np.float64), Z64)
    bound = np.concatenate([tol_kernel + tol_solve, [E[:, 0].sum() + 2.0 ** -23 * abs(ref[-1])]])
    assert np.all(np.abs(g - ref) <= bound), (g, ref, bound)
    # the oracle's estimator against the exact gradient (dense trace): the
    # probes' own noise, reported
    _, exact = oracle.mll_exact(h, X64, p.y.astype(np.float64))
    print("grad gpu   ", np.array2string(g, precision=4))
    print("grad oracle", np.array2string(ref, precision=4))
    print("grad exact ", np.array2string(exact, precision=4))
    print(f"|gpu - estimator| / bound max {np.max(np.abs(g - ref) / bound):.3f}; "
          f"|estimator - exact| / |exact| = {np.linalg.norm(ref - exact) / np.linalg.norm(exact):.3e}; "
          f"epochs {info['epochs']}")
    # data fit 1/2 y^T u: off by at most 1/2 |y|^T |E_0| (+ FP32 rounding of u)
    fit = 0.5 * float(B64[:, 0] @ Wstar[:, 0])
    assert abs(info["data_fit"] - fit) <= 0.5 * float(np.abs(B64[:, 0]) @ (E[:, 0] + 2.0 ** -23 * np.abs(W[:, 0])))
    ap.ap_destroy(ctx)
