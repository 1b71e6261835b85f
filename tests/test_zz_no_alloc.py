"""ap_grad_quadforms_static: the allocation-free variant of the MLL-gradient
quadratic forms, for callers that must not allocate device memory in their
steady state (under stream capture, in latency-bound serving loops, or when
their own pool owns the free HBM).  Checked through the C ABI against
ap_grad_quadforms on the same inputs, on two calls in a row (the fixed scratch
is reused and must not carry state from one call to the next).

Kept in a file collected last, so that a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_2310_17137_gb300 as ap
import workloads as wl

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")


@pytest.mark.parametrize("n,d,c,kern", [(3000, 5, 16, wl.MATERN52), (1500, 11, 4, wl.RBF), (777, 3, 1, wl.MATERN32)])
def test_static_matches_allocating_entry_point_twice(n, d, c, kern):
    p = wl.random_problem(n, d, 256, c, kern, 0.05, 11)
    ctx = ap.ap_create(_t(p.X), ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise),
                       ap.ap_opts_default(block=p.block))
    rng = np.random.default_rng(12)
    U = rng.standard_normal((n, c)).astype(np.float32)
    V = rng.standard_normal((n, c)).astype(np.float32)
    alpha = rng.uniform(-1, 1, c)
    ref = ap.ap_grad_quadforms(ctx, _t(U), _t(V), alpha)
    # every derivative of K_hat is non-negative, so the same forms on |U|, |V|, |alpha|
    # bound the size of every term (the scale of the 1e-5 tolerance of the parity tests)
    mag = ap.ap_grad_quadforms(ctx, _t(np.abs(U)), _t(np.abs(V)), np.abs(alpha))
    for _ in range(2):
        g = ap.ap_grad_quadforms_static(ctx, _t(U), _t(V), alpha)
        assert np.all(np.abs(g - ref) <= 1e-5 * mag + 1e-12), (g, ref)
    ap.ap_destroy(ctx)


def test_static_rejects_problems_beyond_the_scratch():
    # n * (d + 2) partials beyond AP_STATIC_SCRATCH_BYTES -> a clear status, no launch
    n, d = 600_000, 32
    X = np.random.default_rng(0).uniform(size=(n, d)).astype(np.float32)
    ctx = ap.ap_create(_t(X), ap.Hyper(ap.AP_RBF, np.full(d, 2.0), 1.0, 0.5), ap.ap_opts_default(block=64))
    U = torch.zeros((n, 32), device="cuda:0")  # c = 32: 128-row blocks, 4688 x 34 partials > 1 MiB
    with pytest.raises(ap.ApError) as e:
        ap.ap_grad_quadforms_static(ctx, U, U, np.ones(32))
    assert e.value.status == ap.AP_ERR_SCRATCH_LIMIT
    ap.ap_destroy(ctx)
