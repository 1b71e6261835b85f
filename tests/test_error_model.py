"""The derived error bounds of tests/error_model.py, checked on the CPU against
an emulation of the tensor-core form's arithmetic (FP16 hi/lo distance
operands with FP32 accumulation, BF16 hi/lo kernel values and Delta, FP32
epilogue) running Alg. 1: the emulation must stay inside the bounds at every
step, and planted mistakes in it (a dropped product, a perturbed lengthscale, a
missing noise diagonal) must break them.  This pins the bound itself; the GPU
tests then hold the kernels to it.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from error_model import LOG2E, R_ROUND, TcErrorModel, scaled_inputs

F32 = np.float32


def bf16(v):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    v = np.asarray(v, dtype=F32)
    bits = v.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(F32)


def split16(v):
    v = np.asarray(v, dtype=F32)
    hi = v.astype(np.float16)
    lo = (v - hi.astype(F32)).astype(np.float16)
    return hi.astype(F32), lo.astype(F32)


def emulated_update(p, R, I, delta, mistake=None):
    """R - K_hat(X, X_I) Delta the way the tensor-core kernel computes it."""
    n, b = p.n, p.block
    lo, hi = I * b, min(n, I * b + b)
    ell = np.asarray(p.lengthscale, dtype=np.float64).copy()
    if mistake == "lengthscale":
        ell[0] *= 1.01
    z = scaled_inputs(p.kernel, p.X, ell)
    a = (z * z).sum(axis=1)
    rh, rl = split16(z.astype(F32))
    ch, cl = split16((-2.0 * z[lo:hi]).astype(F32))
    ah, al = split16(a.astype(F32))
    t = np.zeros((n, hi - lo), dtype=F32)
    for k in range(p.d):
        for x, y in ((rh, ch), (rh, cl), (rl, ch)):
            t = (t + np.outer(x[:, k], y[:, k]).astype(F32)).astype(F32)
    for v in (ah, al):
        t = (t + v[:, None]).astype(F32)
    for v in (ah[lo:hi], al[lo:hi]):
        t = (t + v[None, :]).astype(F32)
    if p.kernel == wl.RBF:
        P = np.exp2(-t).astype(F32)
    else:
        u = np.sqrt(np.abs(t)).astype(F32)
        e = np.exp2(-u).astype(F32)
        if p.kernel == wl.MATERN32:
            poly = (u * F32(1 / LOG2E) + F32(1)).astype(F32)
        else:
            poly = ((u * F32(1 / (3 * LOG2E ** 2)) + F32(1 / LOG2E)).astype(F32) * u + F32(1)).astype(F32)
        P = (poly * e).astype(F32)
    P_hi = bf16(P)
    P_lo = bf16(P - P_hi)
    d32 = delta.astype(F32)
    d_hi = bf16(d32)
    d_lo = bf16(d32 - d_hi)
    acc = (P_hi @ d_hi).astype(F32) + (P_hi @ d_lo).astype(F32)
    if mistake != "drop_lo":
        acc = (acc + (P_lo @ d_hi).astype(F32)).astype(F32)
    out = (R.astype(np.float64) - float(p.outputscale) * acc.astype(np.float64)).astype(F32)
    if mistake != "no_noise":
        diag = slice(lo, hi)
        out[diag] = (out[diag].astype(np.float64) - float(p.noise) * d32.astype(np.float64)).astype(F32)
    return out


def run_checks(p, k, mistake=None):
    """Alg. 1 with the emulated update; returns the largest ratio of an update
    error to its bound (per step on the chosen rows, and on all rows at the end)."""
    em = TcErrorModel(p, kdp=(3 * p.d + 4 + 15) // 16 * 16)
    h, X, B = em.h, em.X, np.asarray(p.B, dtype=np.float64)
    n, b, c = p.n, p.block, p.c
    m = -(-n // b)
    W = np.zeros((n, c), dtype=F32)
    R = B.astype(F32)
    A = np.zeros((n, c))
    SR = np.abs(B)
    worst = 0.0
    for _ in range(k):
        norms = [np.sum(R[J * b:min(n, J * b + b)].astype(np.float64) ** 2) for J in range(m)]
        I = int(np.argmax(norms))
        rows = np.arange(I * b, min(n, I * b + b))
        beta_I = em.beta(A, rows) + R_ROUND * SR[rows]
        e_I = oracle.residual_rows(h, X, B, W.astype(np.float64), rows=rows) - R[rows]
        worst = max(worst, float(np.max(np.abs(e_I) / beta_I)))
        K = oracle.gram(h, X[rows], X[rows], row0=rows[0], col0=rows[0])
        delta = oracle.chol_solve(oracle.cholesky(K), R[rows].astype(np.float64)).astype(F32)
        W_new = W.copy()
        W_new[rows] = (W[rows] + delta).astype(F32)
        A[rows] += np.abs(W_new[rows].astype(np.float64) - W[rows])
        R = emulated_update(p, R, I, delta.astype(np.float64), mistake)
        W = W_new
        SR += np.abs(R)
    beta = em.beta(A) + R_ROUND * SR
    e = oracle.residual_rows(h, X, B, W.astype(np.float64)) - R
    return max(worst, float(np.max(np.abs(e) / beta)))


CASES = [(600, 3, 128, 4, wl.MATERN52), (500, 11, 128, 4, wl.RBF), (450, 6, 96, 3, wl.MATERN32)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}d{c[1]}k{c[4]}")
def test_emulated_tc_arithmetic_stays_inside_the_bound(case):
    n, d, b, c, kern = case
    p = wl.random_problem(n, d, b, c, kern, 0.05, 31)
    m = -(-n // b)
    ratio = run_checks(p, 2 * m + 1)
    # inside, and not vacuous: the modelled arithmetic uses a visible part of it
    assert 1e-3 < ratio <= 1.0, ratio


@pytest.mark.parametrize("mistake", ["drop_lo", "lengthscale", "no_noise"])
def test_planted_mistakes_break_the_bound(mistake):
    p = wl.random_problem(600, 3, 128, 4, wl.MATERN52, 0.05, 31)
    assert run_checks(p, 5, mistake) > 1.0
