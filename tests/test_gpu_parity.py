"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances follow from the FP32 arithmetic of the kernels: each kernel entry
carries a relative error of a few units of 2^-24 (ex2.approx / sqrt.approx
are specified to about 2 ulp), and every product sums up to n terms in FP32.
For an output o_i = b_i - sum_j K_ij v_j we therefore bound
    |o_gpu - o_fp64| <= TOL_PROD * (sum_j |K_ij| |v_j| + |b_i|),
TOL_PROD = 2e-5 (about 16 * sqrt(n) ulp at the sizes tested).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2310_17137_gb300 as ap
import workloads as wl

pytestmark = pytest.mark.gpu
TOL_PROD = 2e-5

CASES = [
    # n, d, b, c, kernel   -- several 64-row tiles, ragged last block, padded c and d
    (1000, 3, 256, 1, wl.RBF),
    (1337, 5, 300, 3, wl.MATERN52),
    (2100, 11, 512, 16, wl.RBF),
    (777, 17, 128, 5, wl.MATERN32),
    (513, 1, 64, 32, wl.MATERN52),
]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")


def _hyper(p):
    return ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean)


def _problem(case, seed=0):
    n, d, b, c, kern = case
    return wl.random_problem(n, d, b, c, kern, 0.05, seed)


def _ctx(p, trace_cap=0, **kw):
    opts = ap.ap_opts_default(block=p.block, **kw)
    return ap.ap_create(_t(p.X), _hyper(p), opts, trace_cap=trace_cap)


def _f64(a):
    return np.asarray(a, dtype=np.float64)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}d{c[1]}b{c[2]}c{c[3]}k{c[4]}")
def test_residual_matches_oracle(case):
    p = _problem(case)
    h = oracle.Hyper.of(p)
    rng = np.random.default_rng(1)
    W = rng.standard_normal(p.B.shape).astype(np.float32)
    ctx = _ctx(p)
    R = ap.ap_residual(ctx, _t(p.B), _t(W)).cpu().numpy()
    X64 = _f64(p.X)
    Rref = oracle.residual_rows(h, X64, _f64(p.B), _f64(W))
    K = oracle.gram(h, X64)
    bound = TOL_PROD * (np.abs(K) @ np.abs(_f64(W)) + np.abs(_f64(p.B)))
    assert np.all(np.abs(R - Rref) <= bound), np.max(np.abs(R - Rref) / bound)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}d{c[1]}b{c[2]}c{c[3]}k{c[4]}")
def test_compensated_residual_matches_oracle(case):
    # double-float FP32 recompute: entries to ~1e-11, so the only visible error
    # is the final rounding of each output to FP32 (plus a 1e-9 margin on the sum)
    p = _problem(case, seed=3)
    h = oracle.Hyper.of(p)
    W = np.random.default_rng(5).standard_normal(p.B.shape).astype(np.float32)
    ctx = _ctx(p, residual_mode=ap.AP_RESID_COMPENSATED)
    R = ap.ap_residual(ctx, _t(p.B), _t(W)).cpu().numpy()
    X64 = _f64(p.X)
    Rref = oracle.residual_rows(h, X64, _f64(p.B), _f64(W))
    K = oracle.gram(h, X64)
    bound = 2.0 ** -23 * np.abs(Rref) + 1e-9 * (np.abs(K) @ np.abs(_f64(W)) + np.abs(_f64(p.B)))
    assert np.all(np.abs(R - Rref) <= bound), np.max(np.abs(R - Rref) / bound)


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: f"n{c[0]}d{c[1]}k{c[4]}")
def test_predict_mean_matches_oracle(case):
    p = _problem(case)
    h = oracle.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, mean=0.25)
    w = np.random.default_rng(2).standard_normal(p.n).astype(np.float32)
    Xt = wl.test_points(p, m=333)
    ctx = _ctx(p)
    ap.ap_set_hyper(ctx, ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, 0.25))
    mu = ap.ap_predict_mean(ctx, _t(w), _t(Xt)).cpu().numpy()
    ref = oracle.predict_mean(h, _f64(p.X), _f64(w), _f64(Xt))
    Ks = oracle.gram(h, _f64(Xt), _f64(p.X), noise=False)
    bound = TOL_PROD * (np.abs(Ks) @ np.abs(_f64(w)) + 0.25)
    assert np.all(np.abs(mu - ref) <= bound), np.max(np.abs(mu - ref) / bound)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}d{c[1]}b{c[2]}c{c[3]}k{c[4]}")
def test_ap_steps_match_oracle_replay(case):
    # Run k steps on the GPU, replay the GPU's block sequence in the FP64
    # oracle, compare W element by element and check every GPU choice was a
    # Gauss-Southwell argmax of the oracle's block norms (up to FP32 noise).
    p = _problem(case)
    m = -(-p.n // p.block)
    k = 2 * m + 3
    ctx = _ctx(p, trace_cap=k, tol=1e-30, min_epochs=0, max_steps=k)
    st, W, info, trace = ap.ap_solve(ctx, _t(p.B))
    assert st == ap.AP_ERR_NOT_CONVERGED and info["steps"] == k and len(trace) == k
    W = W.cpu().numpy()
    h = oracle.Hyper.of(p)
    r = oracle.ap_solve(h, _f64(p.X), _f64(p.B), p.block, select=oracle.SEL_FORCED, forced=trace,
                        max_steps=k, trace_cap=k)
    np.testing.assert_array_equal(r.trace, trace)
    assert np.all(r.chosen_norm >= r.max_norm * (1 - 1e-4))
    scale = np.abs(r.W).max()
    assert np.abs(W - r.W).max() <= 2e-4 * scale, np.abs(W - r.W).max() / scale


def test_single_block_is_one_exact_step():
    p = wl.random_problem(700, 4, 1024, 2, wl.RBF, 0.1, 3)
    ctx = _ctx(p, tol=1e-30, min_epochs=0, max_steps=1)
    st, W, info, _ = ap.ap_solve(ctx, _t(p.B))
    Wstar = oracle.dense_solve(oracle.Hyper.of(p), _f64(p.X), _f64(p.B))
    assert info["steps"] == 1
    assert np.linalg.norm(W.cpu().numpy() - Wstar) <= 1e-4 * np.linalg.norm(Wstar)


def test_small_rbf_fp32_solution_error():
    # n = 4096, d = 8, RBF l = 0.5, noise 0.1, 8 blocks of 512, one RHS, tol 1e-6:
    # relative solution error <= 1e-5 against the FP64 dense Cholesky solve.
    p = wl.small_rbf()
    ctx = _ctx(p, tol=1e-6, stop=ap.AP_STOP_MAX_REL, max_epochs=200000)
    st, W, info, _ = ap.ap_solve(ctx, _t(p.B))
    print("small_rbf FP32:", info["epochs"], "epochs", info["refinements"], "refinements",
          info["t_solve_s"], "s", info["rel_res_true"])
    assert st == ap.AP_OK, info
    W = W.cpu().numpy().astype(np.float64)
    h = oracle.Hyper.of(p)
    Wstar = oracle.dense_solve(h, _f64(p.X), _f64(p.B))
    err = np.linalg.norm(W - Wstar) / np.linalg.norm(Wstar)
    R = oracle.residual_rows(h, _f64(p.X), _f64(p.B), W)
    rel = np.linalg.norm(R) / np.linalg.norm(p.B)
    print(f"small_rbf FP32: rel solution error {err:.3e}, true rel residual {rel:.3e}")
    assert err <= 1e-5, err
    assert rel <= 1.05e-6


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}d{c[1]}c{c[3]}k{c[4]}")
def test_grad_quadforms_match_oracle(case):
    p = _problem(case)
    h = oracle.Hyper.of(p)
    rng = np.random.default_rng(4)
    U = rng.standard_normal(p.B.shape).astype(np.float32)
    V = rng.standard_normal(p.B.shape).astype(np.float32)
    alpha = rng.uniform(-1, 1, p.c)
    ctx = _ctx(p)
    g = ap.ap_grad_quadforms(ctx, _t(U), _t(V), alpha)
    X64 = _f64(p.X)
    ref = oracle.grad_quadforms(h, X64, _f64(U), _f64(V), alpha)
    mag = oracle.grad_quadforms(h, X64, np.abs(_f64(U)), np.abs(_f64(V)), np.abs(alpha))
    assert np.all(np.abs(g - ref) <= 1e-5 * mag + 1e-12), (g, ref, mag)


def test_mll_grad_matches_oracle_estimator():
    p = wl.random_problem(600, 3, 600, 1, wl.MATERN32, 0.1, 5)  # one block: exact solves
    l = 7
    Z = wl.rademacher(p.n, l, 5)
    h = oracle.Hyper.of(p)
    ref = oracle.mll_grad_stochastic(h, _f64(p.X), _f64(p.y), _f64(Z))
    ctx = _ctx(p, tol=1e-5, stop=ap.AP_STOP_MAX_REL, min_epochs=1)
    st, g, info = ap.ap_mll_grad(ctx, _t(p.y), l, _t(Z))
    assert st == ap.AP_OK
    np.testing.assert_allclose(g, ref, rtol=2e-3, atol=2e-3 * np.abs(ref).max())
    # data fit 1/2 y^T K^-1 y
    u = oracle.dense_solve(h, _f64(p.X), _f64(p.y))
    assert info["data_fit"] == pytest.approx(0.5 * float(_f64(p.y) @ u), rel=1e-4)


def _splitmix64(seed, idx):
    M = (1 << 64) - 1
    z = (seed + (idx + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_cyclic_and_random_selection():
    p = wl.random_problem(900, 3, 128, 2, wl.RBF, 0.1, 6)
    m = -(-p.n // p.block)
    k = 17
    ctx = _ctx(p, trace_cap=k, select=ap.AP_SEL_CYCLIC, tol=1e-30, min_epochs=0, max_steps=k)
    _, _, _, tr = ap.ap_solve(ctx, _t(p.B))
    np.testing.assert_array_equal(tr, np.arange(k) % m)
    seed = 12345
    ctx = _ctx(p, trace_cap=k, select=ap.AP_SEL_RANDOM, seed=seed, tol=1e-30, min_epochs=0, max_steps=k)
    _, W, _, tr = ap.ap_solve(ctx, _t(p.B))
    expect = [((_splitmix64(seed, j) >> 32) * m) >> 32 for j in range(k)]
    np.testing.assert_array_equal(tr, expect)
    r = oracle.ap_solve(oracle.Hyper.of(p), _f64(p.X), _f64(p.B), p.block, select=oracle.SEL_FORCED,
                        forced=tr, max_steps=k)
    assert np.abs(W.cpu().numpy() - r.W).max() <= 2e-4 * np.abs(r.W).max()


def test_not_spd_is_reported():
    X = np.zeros((300, 2), dtype=np.float32)
    with pytest.raises(ap.ApError) as e:
        ap.ap_create(_t(X), ap.Hyper(ap.AP_RBF, [1.0, 1.0], 1.0, 0.0), ap.ap_opts_default(block=128))
    assert e.value.status == ap.AP_ERR_NOT_SPD


def test_warm_start_resumes():
    # checkpoint / resume: a solve started from W0 continues from R = B - K W0
    p = wl.random_problem(1200, 4, 256, 4, wl.MATERN52, 0.1, 8, ell_range=(0.1, 0.3))
    ctx = _ctx(p, tol=1e-30, min_epochs=0, max_steps=7)
    _, W7, _, _ = ap.ap_solve(ctx, _t(p.B))
    ctx2 = _ctx(p, tol=1e-5, stop=ap.AP_STOP_MAX_REL, min_epochs=1, max_epochs=300)
    st, W, info, _ = ap.ap_solve(ctx2, _t(p.B), W0=W7)
    assert st == ap.AP_OK
    R = oracle.residual_rows(oracle.Hyper.of(p), _f64(p.X), _f64(p.B), _f64(W.cpu().numpy()))
    assert np.max(np.linalg.norm(R, axis=0) / np.linalg.norm(p.B, axis=0)) <= 2e-5


@pytest.mark.parametrize("kern", [wl.RBF, wl.MATERN32, wl.MATERN52])
def test_cache_phi_fp64_matches_libm(kern):
    # The cache builds K_II with its own FP64 exp (table-driven, Tang 1989) and
    # Newton-refined sqrt.  Against the host libm on identical r^2: the exp and
    # the polynomial contribute a few ulp, and the sqrt's last-bit error moves
    # e^-u by a relative u * 2^-53 (the conditioning of e^-u), so
    # |phi_gpu - phi| <= (6 + u) 2^-53 phi wherever phi is a normal double.
    rng = np.random.default_rng(7)
    r2 = np.concatenate([[0.0, 1e-300, 1e-40, 1e-30, 1e-12, 1e-6, 0.5, 1.0, 2.0, 1e3, 1e5, 1e13],
                         10.0 ** rng.uniform(-8, 5, 20000), rng.uniform(0, 50, 20000)])
    got = ap.ap_phi_fp64_eval(kern, r2)
    if kern == wl.RBF:
        u = np.zeros_like(r2)
        ref = np.exp(-0.5 * r2)
    elif kern == wl.MATERN32:
        u = np.sqrt(3.0 * r2)
        ref = (1.0 + u) * np.exp(-u)
    else:
        u = np.sqrt(5.0 * r2)
        ref = (1.0 + u + u * u / 3.0) * np.exp(-u)
    if kern == wl.RBF:
        u = 0.5 * r2  # e^{-x}: the rounding of x = r^2/2 is shared, the reduction is exact to x 2^-53
    normal = ref > 1e-300
    bound = (6.0 + u) * 2.0 ** -53 * ref
    assert np.all(np.abs(got - ref)[normal] <= bound[normal]), np.max((np.abs(got - ref) / bound)[normal])
    assert np.all(got[~normal] <= 1e-290) and np.all(got >= 0)
    assert got[0] == 1.0


def test_sfu_rates_are_plausible():
    # per-SM-clock rates of the probe; exp2 runs at least as fast as sqrt on
    # every NVIDIA part, and neither exceeds the 128 lanes of an SM
    e, q = ap.ap_sfu_rates()
    assert 4.0 <= q <= 1.05 * e <= 1.05 * 128.0, (e, q)


@pytest.mark.parametrize("n,d,b,kern,ell", [(1500, 5, 512, wl.MATERN52, (0.3, 3.0)),
                                             (4096, 3, 2048, wl.RBF, (0.05, 0.2))])
def test_tensor_core_cache_matches_fp64_cache(n, d, b, kern, ell):
    # The trailing updates of the FP64 block Cholesky run either as FP64 FMAs or
    # as exact integer slice products on the tensor cores; both caches hold the
    # FP32-rounded inverse factor of nearly the same FP64 factor.  Each run of
    # the same cyclic AP steps is within the FP32 form's replay bound of the
    # exact iterate (2e-4 max|W|, test_ap_steps_match_oracle_replay), so the two
    # agree to twice that.  (The bound presumes moderately conditioned blocks:
    # FP32 inverse factors of a block with condition number kappa differ by up
    # to kappa 2^-24 in the block solve, whichever FP64 factor they come from.)
    # The second case factors blocks of 32 x 32 tiles with a ragged last block.
    p = wl.random_problem(n, d, b, 4, kern, 0.01, 31, ell_range=ell)
    m = -(-n // b)
    Ws = []
    for mode in (ap.AP_CACHE_TC_EXACT, ap.AP_CACHE_FP64):
        opts = ap.ap_opts_default(block=b, select=ap.AP_SEL_CYCLIC, tol=1e-30, min_epochs=0, max_steps=3 * m,
                                  cache_gemm=mode)
        ctx = ap.ap_create(_t(p.X), ap.Hyper(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean), opts)
        st, W, info, _ = ap.ap_solve(ctx, _t(p.B))
        assert info["steps"] == 3 * m
        Ws.append(W.cpu().numpy().astype(np.float64))
        ap.ap_destroy(ctx)
    scale = np.abs(Ws[1]).max()
    assert np.abs(Ws[0] - Ws[1]).max() <= 4e-4 * scale, np.abs(Ws[0] - Ws[1]).max() / scale


@pytest.mark.parametrize("prec", [ap.AP_FP32, ap.AP_BF16_REFINE], ids=["fp32", "bf16"])
def test_solve_host_equals_device_solve(prec):
    # the one-shot host-buffer entry point runs the same deterministic solve as
    # ap_create + ap_solve on device copies of the same inputs
    p = wl.random_problem(3000, 6, 512, 4, wl.MATERN52, 0.05, 47)
    opts = dict(block=p.block, precision=prec, tol=1e-4, stop=ap.AP_STOP_MAX_REL, min_epochs=1, max_epochs=200,
                refine_every=4)
    st_h, W_h, info_h = ap.ap_solve_host(p.X, p.B, _hyper(p), ap.ap_opts_default(**opts))
    ctx = _ctx(p, **{k: v for k, v in opts.items() if k != "block"})
    st_d, W_d, info_d, _ = ap.ap_solve(ctx, _t(p.B))
    assert st_h == st_d and info_h["epochs"] == info_d["epochs"]
    np.testing.assert_array_equal(W_h, W_d.cpu().numpy())
    ap.ap_destroy(ctx)
