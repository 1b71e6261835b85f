"""ap_grad_quadforms_static: the allocation-free variant of the MLL-gradient
quadratic forms.  It serves callers that cannot let a library allocate device
memory once their steady state has begun: latency-bound serving loops, where
cudaMalloc and cudaFree would synchronise the whole device, and processes whose
own memory pool already holds the free HBM.  Checked through the C ABI against
ap_grad_quadforms on the same inputs, on two calls in a row (the fixed scratch
is reused and must not carry state from one call to the next), and checked to
allocate nothing: neither the context's device bytes nor the device's free
memory change across calls.

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


def _inputs(n, c, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n, c)).astype(np.float32)
    V = rng.standard_normal((n, c)).astype(np.float32)
    return U, V, rng.uniform(-1, 1, c)


# (n=2000, d=32, c=32) takes the one-row-per-thread form of the kernel
# (D + c > 40: 128 rows per CTA) and the widest output, d + 2 = 34 sums
@pytest.mark.parametrize("n,d,c,kern", [(3000, 5, 16, wl.MATERN52), (1500, 11, 4, wl.RBF), (777, 3, 1, wl.MATERN32),
                                        (2000, 32, 32, wl.MATERN52)])
def test_static_matches_allocating_entry_point_twice(n, d, c, kern):
    p = wl.random_problem(n, d, 256, c, kern, 0.05, 11)
    ctx = ap.ap_create(_t(p.X), ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise),
                       ap.ap_opts_default(block=p.block))
    U, V, alpha = _inputs(n, c, 12)
    ref = ap.ap_grad_quadforms(ctx, _t(U), _t(V), alpha)
    # every derivative of K_hat is non-negative, so the same forms on |U|, |V|, |alpha|
    # bound the size of every term (the scale of the 1e-5 tolerance of the parity tests)
    mag = ap.ap_grad_quadforms(ctx, _t(np.abs(U)), _t(np.abs(V)), np.abs(alpha))
    for _ in range(2):
        g = ap.ap_grad_quadforms_static(ctx, _t(U), _t(V), alpha)
        assert np.all(np.abs(g - ref) <= 1e-5 * mag + 1e-12), (g, ref)
    ap.ap_destroy(ctx)


def test_static_on_a_fresh_context_allocates_nothing():
    # the static call comes first on this context: no allocating call has grown
    # its work buffers beforehand
    n, d, c = 4000, 8, 16
    p = wl.random_problem(n, d, 512, c, wl.RBF, 0.05, 13)
    ctx = ap.ap_create(_t(p.X), ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise),
                       ap.ap_opts_default(block=p.block))
    U, V, alpha = _inputs(n, c, 14)
    Ud, Vd = _t(U), _t(V)
    torch.cuda.synchronize()
    # the first call of the process on this device may load the module and look up
    # the scratch array; the steady state starts after it
    first = ap.ap_grad_quadforms_static(ctx, Ud, Vd, alpha)
    torch.cuda.synchronize()
    bytes0, free0 = ap.ap_device_bytes(ctx), torch.cuda.mem_get_info()[0]
    outs = [ap.ap_grad_quadforms_static(ctx, Ud, Vd, alpha) for _ in range(2)]
    torch.cuda.synchronize()
    assert ap.ap_device_bytes(ctx) == bytes0
    assert torch.cuda.mem_get_info()[0] == free0
    ref = ap.ap_grad_quadforms(ctx, Ud, Vd, alpha)
    mag = ap.ap_grad_quadforms(ctx, _t(np.abs(U)), _t(np.abs(V)), np.abs(alpha))
    for g in [first] + outs:
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
