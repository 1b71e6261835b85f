"""Pins of the FP64 oracle against things other than itself.

Each test checks one oracle function against a closed form, a brute-force
computation, an independent library routine or a theorem of the paper, chosen
so that a plausible slip (a dropped term, a wrong sign, a transposed operand, a
wrong index or a missing row) fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.special as sps
import scipy.stats as st

import oracle
from oracle import Hyper
import workloads as wl

KERNELS = [oracle.RBF, oracle.MATERN32, oracle.MATERN52]


def matern_bessel(nu: float, r: float) -> float:
    """General Matern correlation 2^(1-nu)/Gamma(nu) (sqrt(2 nu) r)^nu K_nu(sqrt(2 nu) r)."""
    if r == 0.0:
        return 1.0
    z = math.sqrt(2.0 * nu) * r
    return 2.0 ** (1.0 - nu) / sps.gamma(nu) * z ** nu * sps.kv(nu, z)


# ----------------------------------------------------------------- kernel values

@pytest.mark.parametrize("r", [0.0, 0.05, 0.3, 1.0, 1.7, 3.0, 6.0])
@pytest.mark.parametrize("s", [1.0, 0.37])
def test_matern_values_match_bessel_definition(r, s):
    # 1-D pair at scaled distance r: the half-integer closed forms must equal the
    # Bessel-function definition of the Matern family.
    ell = 0.8
    for kind, nu in [(oracle.MATERN32, 1.5), (oracle.MATERN52, 2.5)]:
        h = Hyper(kind, [ell], s, 0.0)
        got = oracle.kernel_value(h, [0.1], [0.1 + r * ell])
        assert got == pytest.approx(s * matern_bessel(nu, r), rel=1e-12, abs=1e-300)


def test_rbf_is_matern_limit():
    # As nu grows the Matern family tends to the squared exponential.
    h = Hyper(oracle.RBF, [1.0], 1.0, 0.0)
    for r in [0.3, 1.0, 2.0]:
        rbf = oracle.kernel_value(h, [0.0], [r])
        assert abs(matern_bessel(60.0, r) - rbf) < 0.02
        assert abs(matern_bessel(60.0, r) - rbf) < abs(matern_bessel(2.5, r) - rbf)


def test_rbf_ard_matches_gaussian_density():
    # exp(-r^2/2) with r = ||(x-x')/l|| equals the N(x'; diag(l^2)) density up to
    # its normaliser: pins the per-dimension lengthscale scaling.
    rng = np.random.default_rng(7)
    for d in [1, 3, 8, 11]:
        ell = np.exp(rng.uniform(-1.5, 1.0, d))
        s = 1.3
        h = Hyper(oracle.RBF, ell, s, 0.0)
        for _ in range(5):
            x, xp = rng.normal(size=d), rng.normal(size=d)
            dens = st.multivariate_normal(mean=xp, cov=np.diag(ell ** 2)).pdf(x)
            ref = s * dens * (2 * math.pi) ** (d / 2) * np.prod(ell)
            assert oracle.kernel_value(h, x, xp) == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("kind", KERNELS)
def test_kernel_at_zero_and_far(kind):
    h = Hyper(kind, [0.5, 2.0, 1.0], 2.5, 0.0)
    x = np.array([0.3, -1.0, 4.0])
    assert oracle.kernel_value(h, x, x) == pytest.approx(2.5, rel=1e-15)
    assert oracle.kernel_value(h, x, x + 200.0) < 1e-30


@pytest.mark.parametrize("kind", KERNELS)
def test_matern_ard_equals_isotropic_on_rescaled_inputs(kind):
    # k_l(x, x') == k_1(x/l, x'/l): the ARD scaling is a pure input rescaling.
    rng = np.random.default_rng(3)
    d = 5
    ell = np.exp(rng.uniform(-1, 1, d))
    X = rng.normal(size=(6, d))
    h = Hyper(kind, ell, 1.1, 0.0)
    h1 = Hyper(kind, np.ones(d), 1.1, 0.0)
    np.testing.assert_allclose(oracle.gram(h, X, noise=False), oracle.gram(h1, X / ell, noise=False),
                               rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------------ gram

@pytest.mark.parametrize("kind", KERNELS)
def test_gram_symmetric_noise_on_index_diagonal(kind):
    rng = np.random.default_rng(1)
    X = rng.uniform(size=(9, 3))
    X[5] = X[2]  # a duplicated point: noise sits on the index diagonal only
    h = Hyper(kind, [0.4, 0.7, 1.0], 1.0, 0.25)
    K = oracle.gram(h, X)
    np.testing.assert_array_equal(K, K.T)
    np.testing.assert_allclose(np.diag(K), 1.25, rtol=1e-15)
    assert K[2, 5] == pytest.approx(1.0, rel=1e-15)
    Kn = oracle.gram(h, X, noise=False)
    np.testing.assert_allclose(K - Kn, 0.25 * np.eye(9), atol=1e-15)
    # global offsets: a block K_hat(X, X_I) with I = [3, 6) has noise where i == 3 + j
    blk = oracle.gram(h, X, X[3:6], row0=0, col0=3)
    np.testing.assert_allclose(blk, K[:, 3:6], rtol=0, atol=0)
    assert np.all(np.linalg.eigvalsh(K) > 0.2)


# ------------------------------------------------------------- dense solve / Cholesky

def _exact_solve(A, b):
    """Gaussian elimination in exact rational arithmetic on the exact doubles."""
    n = len(b)
    M = [[Fraction(float(A[i, j])) for j in range(n)] + [Fraction(float(b[i]))] for i in range(n)]
    for k in range(n):
        p = max(range(k, n), key=lambda i: abs(M[i][k]))
        M[k], M[p] = M[p], M[k]
        for i in range(k + 1, n):
            f = M[i][k] / M[k][k]
            for j in range(k, n + 1):
                M[i][j] -= f * M[k][j]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = M[i][n] - sum(M[i][j] * x[j] for j in range(i + 1, n))
        x[i] = s / M[i][i]
    return np.array([float(v) for v in x])


@pytest.mark.parametrize("n,kind", [(5, oracle.RBF), (9, oracle.MATERN32), (12, oracle.MATERN52)])
def test_dense_solve_brute_force(n, kind):
    rng = np.random.default_rng(n)
    X = rng.uniform(size=(n, 3))
    y = rng.normal(size=n)
    h = Hyper(kind, [0.5, 0.9, 0.3], 1.2, 0.05)
    K = oracle.gram(h, X)
    exact = _exact_solve(K, y)
    got = oracle.dense_solve(h, X, y)
    np.testing.assert_allclose(got, exact, rtol=1e-11, atol=1e-12 * np.abs(exact).max())


def test_cholesky_matches_lapack_and_reconstructs():
    rng = np.random.default_rng(11)
    X = rng.uniform(size=(300, 4))
    h = Hyper(oracle.MATERN52, [0.3, 0.5, 0.8, 1.1], 1.0, 1e-2)
    K = oracle.gram(h, X)
    L = oracle.cholesky(K)
    np.testing.assert_allclose(L, np.linalg.cholesky(K), rtol=1e-10, atol=1e-12)
    assert np.all(np.triu(L, 1) == 0)
    np.testing.assert_allclose(L @ L.T, K, atol=1e-12)
    B = rng.normal(size=(300, 3))
    np.testing.assert_allclose(oracle.chol_solve(L, B), np.linalg.solve(K, B), rtol=1e-8, atol=1e-10)


def test_cholesky_reports_non_spd_pivot():
    A = np.eye(4)
    A[2, 2] = -1.0
    with pytest.raises(np.linalg.LinAlgError, match="pivot 2"):
        oracle.cholesky(A)


# ------------------------------------------------------------------ block selection

def test_gs_select_block_norms_and_ties():
    # n = 10, b = 4: blocks [0,4), [4,8), [8,10) (the last one short)
    R = np.zeros((10, 2))
    R[1] = [1.0, 2.0]      # block 0: 5
    R[6] = [0.0, 3.0]      # block 1: 9
    R[8] = [2.0, 2.0]      # block 2: 8 ...
    R[9] = [1.0, 0.0]      # ... + 1 = 9 (tie with block 1)
    I, norms = oracle.gs_select(R, 4)
    np.testing.assert_array_equal(norms, [5.0, 9.0, 9.0])
    assert I == 1  # tie goes to the smallest index
    R[9] = [1.0, 0.5]
    assert oracle.gs_select(R, 4)[0] == 2
    # the rule uses the Frobenius norm over all columns, not a per-column GS
    R2 = np.zeros((8, 2))
    R2[0] = [3.0, 0.0]
    R2[4] = [2.5, 2.5]
    assert oracle.gs_select(R2, 4)[0] == 1


# ------------------------------------------------------------------- Alg. 1 pins

def _problem(n=96, d=3, c=2, kind=oracle.MATERN52, noise=0.05, seed=0):
    p = wl.random_problem(n, d, 16, c, kind, noise, seed)
    return Hyper.of(p), p.X.astype(np.float64), p.B.astype(np.float64)


def test_single_block_is_exact_after_one_step():
    # b = n: Alg. 1 is one Cholesky solve of the whole system (Sec. 4).
    h, X, B = _problem(n=80)
    r = oracle.ap_solve(h, X, B, b=80, max_steps=1, trace_cap=1)
    Wstar = np.linalg.solve(oracle.gram(h, X), B)
    np.testing.assert_allclose(r.W, Wstar, rtol=1e-9, atol=1e-10 * np.abs(Wstar).max())
    assert np.abs(r.R).max() < 1e-9 * np.abs(B).max()


@pytest.mark.parametrize("kind", KERNELS)
def test_residual_identity_and_block_zeroing(kind):
    # Residual lemma (App. B): R = B - K W after every update, and R_I = 0 right
    # after block I is updated (Eq. text_update_of_r with K_II K_II^-1 = E).
    h, X, B = _problem(n=70, c=3, kind=kind)
    b = 16  # blocks of 16, the last one has 6 rows
    K = oracle.gram(h, X)
    for steps in [1, 2, 5, 9]:
        r = oracle.ap_solve(h, X, B, b=b, max_steps=steps, trace_cap=steps)
        np.testing.assert_allclose(r.R, B - K @ r.W, atol=1e-11 * np.abs(B).max())
        I = r.trace[-1]
        assert np.abs(r.R[I * b:(I + 1) * b]).max() < 1e-11 * np.abs(B).max()


def test_energy_decrease_is_exact_and_monotone():
    # h(W) = 1/2 tr(W^T K W) - tr(B^T W) drops by exactly 1/2 ||R_I||^2_{K_II^-1}
    # = 1/2 tr(R_I^T Delta) per step (proof of Thm. 1, App. C).
    h, X, B = _problem(n=64, c=2)
    K = oracle.gram(h, X)
    steps = 12
    r = oracle.ap_solve(h, X, B, b=16, max_steps=steps, trace_cap=steps)
    hist = []
    for k in range(1, steps + 1):
        rk = oracle.ap_solve(h, X, B, b=16, max_steps=k)
        hist.append(0.5 * np.trace(rk.W.T @ K @ rk.W) - np.trace(B.T @ rk.W))
    hist = np.array(hist)
    scale = abs(hist).max()
    np.testing.assert_allclose(r.energy, hist, atol=1e-11 * scale)
    prev = np.concatenate([[0.0], hist[:-1]])
    np.testing.assert_allclose(hist - prev, r.pred_dec, atol=1e-11 * scale)
    assert np.all(np.diff(np.concatenate([[0.0], hist])) < 0)


def test_gs_choice_recorded_is_the_argmax():
    h, X, B = _problem(n=90, c=4)
    r = oracle.ap_solve(h, X, B, b=16, max_steps=20, trace_cap=20)
    np.testing.assert_array_equal(r.chosen_norm, r.max_norm)
    # replaying step by step with the block-norm function gives the same choices
    W = np.zeros_like(B)
    R = B.copy()
    K = oracle.gram(h, X)
    for j in range(20):
        I, norms = oracle.gs_select(R, 16)
        assert I == r.trace[j]
        lo, hi = I * 16, min(90, I * 16 + 16)
        D = np.linalg.solve(K[lo:hi, lo:hi], R[lo:hi])
        W[lo:hi] += D
        R -= K[:, lo:hi] @ D
    np.testing.assert_allclose(W, r.W, rtol=1e-9, atol=1e-12)


def test_alternating_projection_equals_block_coordinate_descent():
    # App. B lemma: Alg. 1 and Alg. 2 produce the same iterates for one block sequence.
    h, X, B = _problem(n=75, c=2, kind=oracle.RBF)
    r = oracle.ap_solve(h, X, B, b=16, max_steps=17, trace_cap=17)
    Wb = oracle.bcd(h, X, B, 16, r.trace)
    np.testing.assert_allclose(r.W, Wb, rtol=1e-9, atol=1e-11 * np.abs(Wb).max())
    rng = np.random.default_rng(5)
    seq = rng.integers(0, 5, 13)
    ra = oracle.ap_solve(h, X, B, b=16, select=oracle.SEL_FORCED, forced=seq, max_steps=13,
                         trace_cap=13)
    np.testing.assert_array_equal(ra.trace, seq)
    np.testing.assert_allclose(ra.W, oracle.bcd(h, X, B, 16, seq), rtol=1e-9, atol=1e-11)


def test_cyclic_selection_order():
    h, X, B = _problem(n=64, c=1)
    r = oracle.ap_solve(h, X, B, b=16, select=oracle.SEL_CYCLIC, max_steps=10, trace_cap=10)
    np.testing.assert_array_equal(r.trace, [0, 1, 2, 3, 0, 1, 2, 3, 0, 1])


@pytest.mark.parametrize("kind", KERNELS)
def test_theorem1_rate_bound(kind):
    # Thm. 1: ||W^(t) - W*||_K^2 <= exp(-t / kappa') ||W*||_K^2, kappa' = max_I
    # lambda_max(K_II) / lambda_min(K); eigenvalues from LAPACK.
    h, X, B = _problem(n=128, c=3, kind=kind, noise=0.1, seed=2)
    b = 32
    K = oracle.gram(h, X)
    lmin = np.linalg.eigvalsh(K)[0]
    lmaxp = max(np.linalg.eigvalsh(K[i:i + b, i:i + b])[-1] for i in range(0, 128, b))
    kp = lmaxp / lmin
    Wstar = np.linalg.solve(K, B)
    e0 = np.trace(Wstar.T @ K @ Wstar)
    for t in range(1, 6):
        r = oracle.ap_solve(h, X, B, b=b, max_steps=t * 4)
        E = r.W - Wstar
        assert np.trace(E.T @ K @ E) <= math.exp(-t / kp) * e0 * (1 + 1e-12)


def test_converges_to_dense_solution_and_stopping_rules():
    h, X, B = _problem(n=100, c=3, noise=0.1)
    Wstar = oracle.dense_solve(h, X, B)
    r = oracle.ap_solve(h, X, B, b=16, tol=1e-10, stop=oracle.STOP_MAX_REL, max_epochs=3000)
    assert r.status == oracle.OK
    assert np.all(r.rel <= 1e-10)
    np.testing.assert_allclose(r.W, Wstar, rtol=1e-7, atol=1e-8 * np.abs(Wstar).max())
    # min epochs: a loose tolerance still runs 11 epochs (Sec. 5)
    r2 = oracle.ap_solve(h, X, B, b=16, tol=10.0)
    assert r2.status == oracle.OK and r2.epochs == 11 and r2.steps == 11 * 7
    # max epochs reached -> not converged
    r3 = oracle.ap_solve(h, X, B, b=16, tol=1e-30, min_epochs=1, max_epochs=3)
    assert r3.status == oracle.NOT_CONVERGED and r3.epochs == 3 and r3.steps == 21
    # the mean rule is strict, the Frobenius rule of Alg. 1 is not
    rm = oracle.ap_solve(h, X, B, b=16, tol=1e-4, stop=oracle.STOP_MEAN_REL, min_epochs=1)
    assert rm.rel.mean() < 1e-4
    rf = oracle.ap_solve(h, X, B, b=16, tol=1e-4, stop=oracle.STOP_FRO, min_epochs=1)
    assert np.linalg.norm(rf.R) <= 1e-4 * np.linalg.norm(B)
    ry = oracle.ap_solve(h, X, B, b=16, tol=1e-4, stop=oracle.STOP_Y_REL, min_epochs=1)
    assert ry.rel[0] <= 1e-4


def test_non_spd_block_is_reported():
    X = np.zeros((8, 2))
    h = Hyper(oracle.RBF, [1.0, 1.0], 1.0, 0.0)  # all points equal, no noise -> singular
    r = oracle.ap_solve(h, X, np.ones((8, 1)), b=4)
    assert r.status == oracle.NOT_SPD and r.bad_block == 0


def test_block_update_rows_subset_matches_full():
    h, X, B = _problem(n=50, c=2)
    D = np.random.default_rng(0).normal(size=(16, 2))
    full = oracle.block_update(h, X, 16, D, B)
    rows = [0, 7, 20, 31, 49]
    sub = oracle.block_update(h, X, 16, D, B, rows=rows)
    np.testing.assert_allclose(sub[rows], full[rows], rtol=0, atol=0)
    K = oracle.gram(h, X)
    np.testing.assert_allclose(full, B - K[:, 16:32] @ D, atol=1e-12)


def test_residual_rows_is_b_minus_kw():
    h, X, B = _problem(n=40, c=2)
    W = np.random.default_rng(1).normal(size=B.shape)
    K = oracle.gram(h, X)
    np.testing.assert_allclose(oracle.residual_rows(h, X, B, W), B - K @ W, atol=1e-12)
    np.testing.assert_allclose(oracle.residual_rows(h, X, B, W, rows=[3, 39]), (B - K @ W)[[3, 39]],
                               atol=1e-12)


# ---------------------------------------------------------------- posterior mean

@pytest.mark.parametrize("kind", KERNELS)
def test_posterior_mean_interpolates_at_zero_noise(kind):
    rng = np.random.default_rng(4)
    X = rng.uniform(size=(25, 2))
    y = np.sin(3 * X[:, 0]) + X[:, 1]
    h = Hyper(kind, [0.6, 0.6], 1.0, 1e-10, mean=0.3)
    w = oracle.dense_solve(h, X, y - h.mean)
    np.testing.assert_allclose(oracle.predict_mean(h, X, w, X), y, atol=1e-5)
    Xs = rng.uniform(size=(7, 2))
    hn = Hyper(kind, [0.6, 0.6], 1.0, 0.0, mean=0.3)
    Ks = oracle.gram(hn, Xs, X, noise=False)
    np.testing.assert_allclose(oracle.predict_mean(h, X, w, Xs), 0.3 + Ks @ w, rtol=1e-12)


# ------------------------------------------------------------------------ MLL

@pytest.mark.parametrize("kind", KERNELS)
def test_mll_value_matches_gaussian_logpdf(kind):
    rng = np.random.default_rng(8)
    X = rng.uniform(size=(40, 3))
    y = rng.normal(size=40)
    h = Hyper(kind, [0.3, 0.8, 1.5], 1.4, 0.07, mean=0.2)
    K = oracle.gram(h, X)
    lp = st.multivariate_normal(mean=np.full(40, 0.2), cov=K).logpdf(y)
    assert oracle.mll_value(h, X, y) == pytest.approx(-lp - 20 * math.log(2 * math.pi), rel=1e-11)


def _with(h: Hyper, p: int, delta: float) -> Hyper:
    ell = h.ell.copy()
    s, noise, mean = h.s, h.noise, h.mean
    d = h.d
    if p < d:
        ell[p] += delta
    elif p == d:
        s += delta
    elif p == d + 1:
        noise += delta
    else:
        mean += delta
    return Hyper(h.kernel, ell, s, noise, mean)


def _theta(h: Hyper, p: int) -> float:
    return list(h.ell) [p] if p < h.d else [h.s, h.noise, h.mean][p - h.d]


@pytest.mark.parametrize("kind", KERNELS)
def test_exact_mll_gradient_matches_central_differences(kind):
    rng = np.random.default_rng(9)
    X = rng.uniform(size=(60, 3))
    y = np.sin(4 * X[:, 0]) + 0.1 * rng.normal(size=60)
    h = Hyper(kind, [0.4, 0.9, 1.7], 1.3, 0.05, mean=0.1)
    _, g = oracle.mll_exact(h, X, y)
    for p in range(h.d + 3):
        t = _theta(h, p)
        step = 1e-5 * max(abs(t), 1.0)
        fd = (oracle.mll_value(_with(h, p, step), X, y) - oracle.mll_value(_with(h, p, -step), X, y)) / (2 * step)
        assert g[p] == pytest.approx(fd, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("kind", KERNELS)
def test_grad_quadforms_match_finite_difference_of_gram(kind):
    rng = np.random.default_rng(10)
    n, c = 30, 3
    X = rng.uniform(size=(n, 2))
    h = Hyper(kind, [0.5, 1.2], 0.8, 0.2)
    U, V = rng.normal(size=(n, c)), rng.normal(size=(n, c))
    alpha = np.array([-0.5, 0.25, 0.25])
    g = oracle.grad_quadforms(h, X, U, V, alpha)
    for p in range(h.d + 2):
        step = 1e-6 * max(abs(_theta(h, p)), 1.0)
        dK = (oracle.gram(_with(h, p, step), X) - oracle.gram(_with(h, p, -step), X)) / (2 * step)
        ref = sum(alpha[k] * U[:, k] @ dK @ V[:, k] for k in range(c))
        assert g[p] == pytest.approx(ref, rel=1e-7, abs=1e-9)


def test_stochastic_gradient_unbiased():
    # Eq. loss_grad_unbiased: the probe average is unbiased for the exact gradient.
    rng = np.random.default_rng(12)
    n = 32
    X = rng.uniform(size=(n, 2))
    y = np.cos(5 * X[:, 1])
    h = Hyper(oracle.MATERN32, [0.4, 0.7], 1.0, 0.1)
    _, gex = oracle.mll_exact(h, X, y)
    reps = []
    for k in range(40):
        Z = 2.0 * np.random.default_rng(100 + k).integers(0, 2, (n, 50)) - 1.0
        reps.append(oracle.mll_grad_stochastic(h, X, y, Z))
    reps = np.array(reps)
    mean, sem = reps.mean(0), reps.std(0, ddof=1) / math.sqrt(len(reps))
    assert np.all(np.abs(mean - gex) <= 4.5 * sem + 1e-9)
    # the data-fit part (mean gradient) has no probe noise at all
    np.testing.assert_allclose(reps[:, -1], gex[-1], rtol=1e-10)
