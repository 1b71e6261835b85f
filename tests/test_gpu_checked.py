"""The bounds-checked build: the same sources compiled with AP_CHECKED into
libap_checked.so, where the kernels check their tile and row indices against
the sizes they were given before the accesses those indices guard.  A failed
check is recorded (translation unit and source line) and the access skipped,
so it never faults.

In a child process with AP_CHECKED=1 (which loads the checked library): the
self-test kernel records an out-of-range read and not an in-range one; then
small odd shapes (n not a multiple of the tile, ragged last blocks, d and c
that need padding, more tiles than SMs so that tiles are split between CTAs)
run through every entry point of the hot path in both forms without a single
failed check, and their results still agree with the FP64 oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
import torch
import oracle
import workloads as wl
import paper_2310_17137_gb300 as ap
from paper_2310_17137_gb300 import _capi

assert _capi.checked() and _capi.lib_path().endswith("libap_checked.so")
torch.cuda.init()
assert ap.ap_bounds_violations()[0] == 0
assert ap.ap_bounds_selftest(7) == ap.AP_OK and ap.ap_bounds_violations()[0] == 0
assert ap.ap_bounds_selftest(8) == ap.AP_OK
n_bad, where = ap.ap_bounds_violations()
assert n_bad == 1 and where.startswith("misc.cu:"), (n_bad, where)
assert ap.ap_bounds_violations()[0] == 0  # cleared by the read

def t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")

def clean(what):
    n_bad, where = ap.ap_bounds_violations()
    assert n_bad == 0, f"{what}: failed index check at {where}"

CASES = [  # n, d, b, c, kernel, form
    (1000, 1, 256, 1, wl.RBF, ap.AP_FP32),
    (1337, 5, 300, 3, wl.MATERN52, ap.AP_BF16_REFINE),
    (777, 17, 192, 32, wl.MATERN32, ap.AP_BF16_REFINE),
    (2100, 20, 512, 5, wl.MATERN52, ap.AP_FP32),
    (20600, 3, 256, 16, wl.MATERN52, ap.AP_BF16_REFINE),
    (20600, 11, 1024, 16, wl.RBF, ap.AP_BF16_REFINE),
]
for n, d, b, c, kern, form in CASES:
    name = f"n{n} d{d} b{b} c{c} kernel {kern} form {form}"
    p = wl.random_problem(n, d, b, c, kern, 0.05, 61)
    h = oracle.Hyper.of(p)
    X64, B64 = p.X.astype(np.float64), p.B.astype(np.float64)
    m = -(-n // b)
    k = 2 * m + 1
    hyper = ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean)
    ctx = ap.ap_create(t(p.X), hyper, ap.ap_opts_default(block=b, precision=form, tol=1e-30, min_epochs=0,
                                                         max_steps=k, refine_every=1), trace_cap=k)
    clean(name + " create")
    st, W, info, trace = ap.ap_solve(ctx, t(p.B))
    assert st == ap.AP_ERR_NOT_CONVERGED and info["steps"] == k, (name, st, info["steps"])
    clean(name + " solve")
    W = W.cpu().numpy().astype(np.float64)
    r = oracle.ap_solve(h, X64, B64, b, select=oracle.SEL_FORCED, forced=trace, max_steps=k, trace_cap=k)
    rel = np.abs(W - r.W).max() / np.abs(r.W).max()
    assert rel <= (2e-4 if form == ap.AP_FP32 else 2e-2), (name, rel)
    R = ap.ap_residual(ctx, t(p.B), t(W)).cpu().numpy()
    clean(name + " residual")
    rows = np.arange(0, n, max(1, n // 97))
    Rref = oracle.residual_rows(h, X64, B64, W, rows=rows)
    scale = np.abs(B64[rows]).max() + np.abs(Rref).max()
    assert np.abs(R[rows] - Rref).max() <= 1e-4 * scale, (name, np.abs(R[rows] - Rref).max() / scale)
    Xt = wl.test_points(p, m=333)
    mu = ap.ap_predict_mean(ctx, t(W[:, 0]), t(Xt)).cpu().numpy()
    clean(name + " predict")
    ref = oracle.predict_mean(h, X64, W[:, 0], Xt.astype(np.float64))
    Ks = oracle.gram(h, Xt.astype(np.float64), X64, noise=False)
    bound = 2e-5 * (np.abs(Ks) @ np.abs(W[:, 0]) + abs(p.mean))
    assert np.all(np.abs(mu - ref) <= bound), (name, np.max(np.abs(mu - ref) / bound))
    if n <= 2100:
        V = np.random.default_rng(3).standard_normal(W.shape)
        alpha = np.linspace(-1.0, 1.0, c)
        q = ap.ap_grad_quadforms(ctx, t(W), t(V), alpha)
        clean(name + " quadforms")
        qref = oracle.grad_quadforms(h, X64, W, V, alpha)
        mag = oracle.grad_quadforms(h, X64, np.abs(W), np.abs(V), np.abs(alpha))
        assert np.all(np.abs(q - qref) <= 1e-4 * mag + 1e-6), name
    ap.ap_destroy(ctx)
    clean(name + " destroy")
    print("clean:", name, f"rel {rel:.1e}", flush=True)
print("CHECKED-OK")
'''


def test_checked_build_odd_shapes_pass_every_index_check():
    env = dict(os.environ, AP_CHECKED="1")
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    print(r.stdout[-3000:])
    assert r.returncode == 0 and "CHECKED-OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
