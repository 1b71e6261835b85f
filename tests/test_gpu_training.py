"""End-to-end hyperparameter training through the MLL-gradient autograd
function (the paper's training loop, Sec. 5: Adam over the stochastic gradient
of Eq. loss_grad_unbiased, every gradient from an AP solve).

Data are drawn from a Matern-5/2 GP with known hyperparameters; training starts
far from them.  The exact negative MLL (dense FP64, oracle) must drop and every
lengthscale must move towards its generating value."""
import numpy as np
import pytest
import torch

import oracle
import paper_2310_17137_gb300 as ap
import workloads as wl

pytestmark = pytest.mark.gpu


def test_adam_over_mll_gradient_improves_exact_mll():
    n, d = 2048, 2
    rng = np.random.default_rng(7)
    X = rng.uniform(0.0, 1.0, (n, d)).astype(np.float32)
    true = oracle.Hyper(wl.MATERN52, [0.15, 0.4], 1.0, 0.05)
    L = np.linalg.cholesky(oracle.gram(true, X.astype(np.float64)))
    y = (L @ rng.standard_normal(n)).astype(np.float32)

    ell0, s0, noise0 = np.array([0.6, 0.6]), 1.0, 0.3
    log_ell = torch.tensor(np.log(ell0), dtype=torch.float64, requires_grad=True)
    log_s = torch.tensor(np.log(s0), dtype=torch.float64, requires_grad=True)
    log_noise = torch.tensor(np.log(noise0), dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(0.0, dtype=torch.float64)
    X_dev = torch.from_numpy(X).to("cuda:0")
    y_dev = torch.from_numpy(y).to("cuda:0")
    opts = ap.ap_opts_default(block=512, tol=1e-3, stop=ap.AP_STOP_MEAN_REL, min_epochs=11, max_epochs=300)
    ctx = ap.ap_create(X_dev, ap.Hyper(wl.MATERN52, ell0, s0, noise0), opts)
    adam = torch.optim.Adam([log_ell, log_s, log_noise], lr=0.1)
    for _ in range(30):
        adam.zero_grad()
        fit = ap.MLLDataFit.apply(ctx, y_dev, wl.MATERN52, log_ell.exp(), log_s.exp(), log_noise.exp(), mu, 15)
        fit.backward()
        assert torch.isfinite(log_ell.grad).all() and torch.isfinite(log_noise.grad)
        adam.step()
    ap.ap_destroy(ctx)

    ell1 = log_ell.exp().detach().numpy()
    h0 = oracle.Hyper(wl.MATERN52, ell0, s0, noise0)
    h1 = oracle.Hyper(wl.MATERN52, ell1, float(log_s.detach().exp()), float(log_noise.detach().exp()))
    nll0 = oracle.mll_value(h0, X, y)
    nll1 = oracle.mll_value(h1, X, y)
    assert nll1 < nll0 - 50.0, (nll0, nll1)
    dist0 = np.abs(np.log(ell0) - np.log(true.ell))
    dist1 = np.abs(np.log(ell1) - np.log(true.ell))
    assert np.all(dist1 < dist0), (ell1, true.ell)
