"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers.  It holds none of the solver's
arithmetic, so both the CUDA path and the FP64 oracle can take their inputs
from here without sharing any of the method.

The workloads stand in for the UCI regression sets of the paper's experiments
(Sec. 5 and Table 1: n from 0.24M to 4.2M, d from 3 to 90, Matern kernels,
standardised labels, noise down to 1e-4..1e-2).  None of those datasets is
reproduced.  Every array is drawn in float64 with NumPy's PCG64 and stored as
float32, so the GPU and the oracle read bit-identical values.

Fixed seed streams: data 0, label noise 1, probes 2, hyperparameters 3,
arrivals 4.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_DATA, SEED_NOISE, SEED_PROBES, SEED_HYPER, SEED_ARRIVALS = 0, 1, 2, 3, 4

RBF, MATERN32, MATERN52 = 0, 1, 2
KERNEL_NAMES = {RBF: "rbf", MATERN32: "matern32", MATERN52: "matern52"}


@dataclasses.dataclass
class Problem:
    """One GP system (K + noise I) W = B with its hyperparameters."""
    name: str
    X: np.ndarray            # n x d float32, row-major
    y: np.ndarray            # n float32
    B: np.ndarray            # n x c float32: [y - mean, z_1 .. z_l]
    kernel: int
    lengthscale: np.ndarray  # d float32
    outputscale: float
    noise: float
    mean: float
    block: int
    tol: float
    Xtest: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def c(self) -> int:
        return self.B.shape[1]


def _rng(seed: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, sub]))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _sine_labels(X: np.ndarray, noise_sd: float, sub: int) -> np.ndarray:
    """Labels sum_j sin(2 pi x_j) + noise_sd * N(0, 1), drawn in float64."""
    eps = _rng(SEED_NOISE, sub).standard_normal(X.shape[0])
    return np.sin(2.0 * np.pi * X.astype(np.float64)).sum(axis=1) + noise_sd * eps


def _standardise(y: np.ndarray) -> np.ndarray:
    return (y - y.mean()) / y.std()


def rademacher(n: int, l: int, sub: int = 0) -> np.ndarray:
    """n x l matrix of +-1 probe vectors (Rademacher, as used for AP in App. E)."""
    z = _rng(SEED_PROBES, sub).integers(0, 2, size=(n, l), dtype=np.int8)
    return (2.0 * z.astype(np.float32) - 1.0).astype(np.float32)


def log_uniform(rng: np.random.Generator, lo: float, hi: float, size) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def small_rbf(n: int = 4096, d: int = 8, block: int = 512, lengthscale: float = 0.5,
              noise: float = 0.1, tol: float = 1e-6, n_probes: int = 0, sub: int = 0) -> Problem:
    """Plain FP32 AP solve: X ~ U[0,1]^d, RBF (lengthscale 0.5, outputscale 1),
    noise 0.1, y = sum_j sin(2 pi x_j) + N(0, 0.1^2), blocks of 512, one RHS,
    tolerance 1e-6.  Labels are used as drawn (prior mean 0)."""
    X = _rng(SEED_DATA, sub).uniform(0.0, 1.0, (n, d))
    y = _sine_labels(X, 0.1, sub)
    B = y[:, None]
    if n_probes:
        B = np.concatenate([B, rademacher(n, n_probes, sub).astype(np.float64)], axis=1)
    return Problem(f"rbf_n{n}_d{d}_b{block}", _f32(X), _f32(y), _f32(B), RBF,
                   _f32(np.full(d, lengthscale)), 1.0, float(np.float32(noise)), 0.0, block, tol)


def matern52_ard(n: int = 262144, d: int = 3, block: int = 4096, n_probes: int = 15,
                 noise: float = 1e-2, tol: float = 1e-3, sub: int = 0) -> Problem:
    """X ~ N(0, I_d), Matern-5/2 ARD with lengthscales log-uniform in [0.3, 3],
    noise 1e-2, B = [y, 15 Rademacher probes], tolerance 1e-3.  y is the sine
    label (noise 0.1) standardised to zero mean and unit variance, prior mean 0."""
    X = _rng(SEED_DATA, sub).standard_normal((n, d))
    ell = log_uniform(_rng(SEED_HYPER, sub), 0.3, 3.0, d)
    y = _standardise(_sine_labels(X, 0.1, sub))
    B = np.concatenate([y[:, None], rademacher(n, n_probes, sub).astype(np.float64)], axis=1)
    return Problem(f"matern52_n{n}_d{d}_b{block}", _f32(X), _f32(y), _f32(B), MATERN52,
                   _f32(ell), 1.0, float(np.float32(noise)), 0.0, block, tol)


def rbf_ard_large(n: int = 2097152, d: int = 11, block: int = 8192, n_probes: int = 15,
                  noise: float = 1e-3, tol: float = 1e-2, sub: int = 0) -> Problem:
    """X ~ U[-1,1]^d, RBF ARD with lengthscales log-uniform in [0.2, 2], noise
    1e-3, B = [y, 15 Rademacher probes], tolerance 1e-2, standardised y."""
    X = _rng(SEED_DATA, sub).uniform(-1.0, 1.0, (n, d))
    ell = log_uniform(_rng(SEED_HYPER, sub), 0.2, 2.0, d)
    y = _standardise(_sine_labels(X, 0.1, sub))
    B = np.concatenate([y[:, None], rademacher(n, n_probes, sub).astype(np.float64)], axis=1)
    return Problem(f"rbf_ard_n{n}_d{d}_b{block}", _f32(X), _f32(y), _f32(B), RBF,
                   _f32(ell), 1.0, float(np.float32(noise)), 0.0, block, tol)


def matern32_grad(n: int = 131072, d: int = 8, block: int = 4096, n_probes: int = 31,
                  noise: float = 0.05, tol: float = 1.0, sub: int = 0) -> Problem:
    """MLL-gradient workload: X ~ U[0,1]^d, Matern-3/2 ARD with lengthscales
    log-uniform in [0.3, 3], noise 0.05, B = [y - mean, 31 Rademacher probes].
    Training tolerance 1 as in the paper's GP training (Sec. 5)."""
    X = _rng(SEED_DATA, sub).uniform(0.0, 1.0, (n, d))
    ell = log_uniform(_rng(SEED_HYPER, sub), 0.3, 3.0, d)
    y = _standardise(_sine_labels(X, 0.1, sub))
    B = np.concatenate([y[:, None], rademacher(n, n_probes, sub).astype(np.float64)], axis=1)
    return Problem(f"matern32_n{n}_d{d}_b{block}", _f32(X), _f32(y), _f32(B), MATERN32,
                   _f32(ell), 1.0, float(np.float32(noise)), 0.0, block, tol)


def random_problem(n: int, d: int, block: int, c: int, kernel: int, noise: float,
                   seed: int, ell_range=(0.3, 3.0), x_dist: str = "uniform",
                   outputscale: float = 1.0) -> Problem:
    """Generic small problem for parity tests: any n, d, b, c and kernel."""
    rng = _rng(SEED_DATA, 1000 + seed)
    if x_dist == "normal":
        X = rng.standard_normal((n, d))
    else:
        X = rng.uniform(0.0, 1.0, (n, d))
    ell = log_uniform(_rng(SEED_HYPER, 1000 + seed), ell_range[0], ell_range[1], d)
    y = _standardise(_sine_labels(X, 0.1, 1000 + seed)) if n > 1 else np.ones(n)
    cols = [y[:, None]]
    if c > 1:
        cols.append(rademacher(n, c - 1, 1000 + seed).astype(np.float64))
    B = np.concatenate(cols, axis=1)
    return Problem(f"rand{seed}_{KERNEL_NAMES[kernel]}_n{n}_d{d}_b{block}_c{c}", _f32(X), _f32(y),
                   _f32(B), kernel, _f32(ell), float(np.float32(outputscale)),
                   float(np.float32(noise)), 0.0, block, 1e-6)


def test_points(p: Problem, m: int = 1024, sub: int = 0) -> np.ndarray:
    """m test inputs drawn from the same distribution family as the training inputs."""
    rng = _rng(SEED_DATA, 500 + sub)
    lo, hi = float(p.X.min()), float(p.X.max())
    return _f32(rng.uniform(lo, hi, (m, p.d)))


@dataclasses.dataclass
class Request:
    """One serving request: a GP solve plus a posterior mean on test points."""
    rid: int
    arrival_s: float
    n: int
    d: int
    kernel: int
    lengthscale: np.ndarray
    outputscale: float
    noise: float
    tol: float
    low_precision: bool
    seed: int


def serving_trace(n_requests: int = 512, rate: float = 40.0, n_lo: int = 2 ** 10,
                  n_hi: int = 2 ** 18, seed_sub: int = 0) -> list:
    """Poisson arrivals at `rate` per second; n log-uniform in [n_lo, n_hi];
    d uniform in {3..20}; RBF or Matern-5/2; lengthscales log-uniform in
    [0.3, 3], outputscale in [0.5, 2], noise in [1e-3, 1e-1]; tolerance drawn
    from {1e-2, 1e-4}; half of the requests ask for the low-precision form."""
    rng = _rng(SEED_ARRIVALS, seed_sub)
    t = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    out = []
    for i in range(n_requests):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.integers(3, 21))
        kern = RBF if rng.uniform() < 0.5 else MATERN52
        ell = _f32(log_uniform(rng, 0.3, 3.0, d))
        s = float(np.float32(log_uniform(rng, 0.5, 2.0, 1)[0]))
        noise = float(np.float32(log_uniform(rng, 1e-3, 1e-1, 1)[0]))
        tol = 1e-2 if rng.uniform() < 0.5 else 1e-4
        low = bool(rng.uniform() < 0.5)
        out.append(Request(i, float(t[i]), n, d, kern, ell, s, noise, tol, low, 10_000 + i))
    return out


def request_data(req: Request, m_test: int = 1024):
    """Training inputs, labels and test inputs of one serving request."""
    rng = _rng(SEED_DATA, req.seed)
    X = rng.uniform(0.0, 1.0, (req.n, req.d))
    y = _standardise(_sine_labels(X, 0.1, req.seed))
    Xt = _rng(SEED_DATA, req.seed + 500_000).uniform(0.0, 1.0, (m_test, req.d))
    return _f32(X), _f32(y), _f32(Xt)


CONFIGS = {
    "small_rbf": small_rbf,
    "matern52_ard": matern52_ard,
    "rbf_ard_large": rbf_ard_large,
    "matern32_grad": matern32_grad,
}
