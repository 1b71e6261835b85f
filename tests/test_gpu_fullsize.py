"""Parity at the full workload sizes, in the launch configuration bench.py
times (same block size, right-hand sides and kernel), on outputs the FP64
oracle can compute one by one: sampled rows of the true residual B - K_hat W.

Bound per sampled output (FP32 recompute): 2e-5 (sum_j |K_ij| |w_j| + |b_i|),
the FP32-product tolerance of the small parity tests; the oracle gives the
magnitude sum through a residual of |W| (all kernel entries are positive).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2310_17137_gb300 as ap
import workloads as wl

pytestmark = pytest.mark.gpu


def _run(p, precision, max_epochs, rows):
    dev = "cuda:0"
    X = torch.from_numpy(p.X).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    ctx = ap.ap_create(X, ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise),
                       ap.ap_opts_default(block=p.block, tol=p.tol, stop=ap.AP_STOP_MAX_REL, min_epochs=1,
                                          max_epochs=max_epochs, precision=precision, refine_every=10))
    st, W, info, _ = ap.ap_solve(ctx, B)
    R = ap.ap_residual(ctx, B, W)
    torch.cuda.synchronize()
    h = oracle.Hyper.of(p)
    X64 = p.X.astype(np.float64)
    W64 = W.cpu().numpy().astype(np.float64)
    ref = oracle.residual_rows(h, X64, p.B.astype(np.float64), W64, rows=rows)
    mag = -oracle.residual_rows(h, X64, np.zeros_like(W64), np.abs(W64), rows=rows)
    got = R.cpu().numpy()[rows]
    bound = 2e-5 * (mag + np.abs(p.B[rows]))
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / bound)
    # the solver's reported residual of column y is the FP32 recompute's
    rel_y = np.linalg.norm(R.cpu().numpy()[:, 0]) / np.linalg.norm(p.B[:, 0])
    assert abs(rel_y - info["rel_res_true"][0]) <= 1e-3 * rel_y + 1e-7
    return info


@pytest.mark.parametrize("precision", [ap.AP_FP32, ap.AP_BF16_REFINE], ids=["fp32", "bf16"])
def test_matern52_n262144_sampled_true_residual(precision):
    p = wl.matern52_ard()
    rows = np.sort(np.random.default_rng(0).choice(p.n, 48, replace=False))
    info = _run(p, precision, max_epochs=2, rows=rows)
    assert info["epochs"] == 2 and info["steps"] == 2 * (p.n // p.block)


@pytest.mark.slow
def test_rbf_n2097152_sampled_true_residual():
    p = wl.rbf_ard_large()
    rows = np.sort(np.random.default_rng(1).choice(p.n, 12, replace=False))
    info = _run(p, ap.AP_BF16_REFINE, max_epochs=1, rows=rows)
    assert info["epochs"] == 1
