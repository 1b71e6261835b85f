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


def _split_tile_rows(n, b, grid, count):
    """Rows of the first `count` 128-row tiles that two persistent CTAs of the
    tensor-core update share (their (tile, chunk) ranges end inside the tile)."""
    tps = -(-b // 128)
    m = -(-n // b)
    nq = -(-b // 128)
    U = m * tps * nq
    rows = []
    for cta in range(1, grid):
        u = U * cta // grid
        if u % nq:
            T = u // nq
            r0 = (T // tps) * b + (T % tps) * 128
            rows.extend(range(r0, min(r0 + 128, n)))
            if len(rows) >= 128 * count:
                break
    return np.asarray(rows, dtype=np.int64)


def test_matern52_n262144_tc_tracked_residual_within_derived_bound():
    """The tensor-core form's own tracked residual after 8 steps of the bench
    configuration (n = 262,144, b = 4096, c = 16), against B - K_hat W of the
    GPU's iterate computed by the oracle, on 48 random rows and the rows of two
    tiles that two CTAs share, under the derived bound of tests/error_model.py.
    In 8 steps no block is chosen twice, so the accumulated |Delta| is |W|."""
    from error_model import R_ROUND, TcErrorModel
    p = wl.matern52_ard()
    k = 8
    dev = "cuda:0"
    X = torch.from_numpy(p.X).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    ctx = ap.ap_create(X, ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise),
                       ap.ap_opts_default(block=p.block, tol=1e-30, min_epochs=0, max_steps=k,
                                          precision=ap.AP_BF16_REFINE, refine_every=0), trace_cap=k)
    st, W, info, trace = ap.ap_solve(ctx, B)
    assert st == ap.AP_ERR_NOT_CONVERGED and info["steps"] == k
    assert len(set(trace.tolist())) == k, trace
    R = ap.ap_tracked_residual(ctx, p.c).cpu().numpy().astype(np.float64)
    W64 = W.cpu().numpy().astype(np.float64)
    grid = torch.cuda.get_device_properties(0).multi_processor_count
    rows = np.unique(np.concatenate([np.random.default_rng(4).choice(p.n, 48, replace=False),
                                     _split_tile_rows(p.n, p.block, grid, 2)]))
    em = TcErrorModel(p, kdp=16)
    A = np.abs(W64)
    KA = em.k_times(A, rows)
    # |R_tau| <= |B| + K_hat A for every tau <= k
    SR = (k + 1) * (np.abs(p.B[rows]) + KA)
    beta = em.beta(A, rows) + R_ROUND * SR
    e = oracle.residual_rows(em.h, em.X, p.B.astype(np.float64), W64, rows=rows) - R[rows]
    assert np.all(np.abs(e) <= beta), np.max(np.abs(e) / beta)
    print(f"tracked residual error / derived bound: max {np.max(np.abs(e) / beta):.3f}")
    ap.ap_destroy(ctx)
