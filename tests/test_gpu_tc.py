"""Parity of the tensor-core form (AP_BF16_REFINE) with the FP64 oracle.

The tensor-core form evaluates the squared distances with FP16 hi/lo operands
(about 22 mantissa bits, FP32 accumulation: absolute error ~ 2^-21 |x_s|^2 in
the exponent argument) and carries kernel values and Delta as BF16 hi/lo pairs
(about 16 bits), so a kernel entry is within ~1e-4 of its FP32 value.  After
2m + 1 steps the iterates of a replay of the GPU's block sequence in the FP64
oracle agree to 5e-3 max|W| (the block solves amplify entry errors by up to
the condition number of K_II; the FP32 form's bound is 2e-4) over up to 2m + 1
steps for a few blocks m.  Accuracy of
whole solves is won back by the FP32 residual recompute (refinement).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2310_17137_gb300 as ap
import workloads as wl

pytestmark = pytest.mark.gpu

CASES = [
    # n, d, b, c, kernel, steps (None: 2m + 1): several 128-row tiles and
    # 128-column chunks, ragged tails; distance operands of K = 16, 32, 64, 48 and
    # 96 (3d + 4 rounded up to 16; d = 30 is the largest the tensor-core form
    # takes, with the largest shared-memory stages at c = 32)
    (1000, 3, 256, 16, wl.MATERN52, None),
    (1337, 5, 300, 3, wl.RBF, None),
    (777, 17, 192, 32, wl.MATERN32, None),
    (2100, 11, 512, 16, wl.RBF, None),
    (900, 30, 384, 32, wl.MATERN52, None),
    # more 128-row tiles than SMs, so the work ranges of the CTAs split tiles
    # between two CTAs (boundary slots).  Nine steps: the differences to the
    # replay grow with the number of steps (each block solve carries the entry
    # errors into W), to about 1.3e-2 max|W| after 2m + 1 = 109..163 steps here,
    # with or without the split
    (20600, 3, 256, 16, wl.MATERN52, 9),
    (20600, 5, 384, 32, wl.RBF, 9),
]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def _ctx(p, trace_cap=0, **kw):
    opts = ap.ap_opts_default(block=p.block, precision=ap.AP_BF16_REFINE, **kw)
    return ap.ap_create(_t(p.X), ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean), opts,
                        trace_cap=trace_cap)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}d{c[1]}b{c[2]}c{c[3]}k{c[4]}")
def test_tc_steps_match_oracle_replay(case):
    n, d, b, c, kern, steps = case
    p = wl.random_problem(n, d, b, c, kern, 0.05, 21)
    m = -(-n // b)
    k = steps or 2 * m + 1
    ctx = _ctx(p, trace_cap=k, tol=1e-30, min_epochs=0, max_steps=k, refine_every=0)
    st, W, info, trace = ap.ap_solve(ctx, _t(p.B))
    assert st == ap.AP_ERR_NOT_CONVERGED and info["steps"] == k
    W = W.cpu().numpy()
    h = oracle.Hyper.of(p)
    r = oracle.ap_solve(h, _f64(p.X), _f64(p.B), b, select=oracle.SEL_FORCED, forced=trace, max_steps=k,
                        trace_cap=k)
    # the GPU's choices are Gauss-Southwell choices of the oracle's norms, up to the form's accuracy
    assert np.all(r.chosen_norm >= r.max_norm * (1 - 2e-2))
    scale = np.abs(r.W).max()
    assert np.abs(W - r.W).max() <= 5e-3 * scale, np.abs(W - r.W).max() / scale


def test_tc_solve_with_refinement_reaches_fp32_accuracy():
    p = wl.random_problem(3000, 5, 256, 16, wl.MATERN52, 0.1, 23, ell_range=(0.1, 0.3))
    ctx = _ctx(p, tol=1e-5, stop=ap.AP_STOP_MAX_REL, min_epochs=1, max_epochs=500, refine_every=3)
    st, W, info, _ = ap.ap_solve(ctx, _t(p.B))
    assert st == ap.AP_OK, info
    assert info["refinements"] >= 1
    R = oracle.residual_rows(oracle.Hyper.of(p), _f64(p.X), _f64(p.B), _f64(W.cpu().numpy()))
    rel = np.linalg.norm(R, axis=0) / np.linalg.norm(p.B, axis=0)
    assert rel.max() <= 1.2e-5, rel
