"""FP64 CPU oracle for the alternating-projection GP solver (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the CUDA path: the C source
``ap_oracle.c`` is compiled with gcc into ``liboracle.so`` and called through
ctypes on float64 NumPy arrays.  Every function states the passage of the paper
it follows (Wu et al., "Large-Scale Gaussian Processes via Alternating
Projection", AISTATS 2024).

Parity status: every function below is pinned by ``tests/test_oracle_pins.py``
against closed forms, brute force or library routines it does not call.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ap_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RBF, MATERN32, MATERN52 = 0, 1, 2
SEL_GS, SEL_CYCLIC, SEL_FORCED = 0, 1, 2
STOP_MEAN_REL, STOP_MAX_REL, STOP_FRO, STOP_Y_REL = 0, 1, 2, 3
OK, NOT_CONVERGED, NOT_SPD, BAD_ARG = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (plain C, -O2, OpenMP over independent rows)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "orc_num_threads": (i32, []),
                "orc_kernel_value": (f64, [i32, i32, P, f64, P, P]),
                "orc_gram": (None, [i32, i32, P, f64, f64, P, i64, i64, P, i64, i64, P]),
                "orc_cholesky": (i64, [i64, P]),
                "orc_chol_solve": (None, [i64, P, i32, P, P]),
                "orc_dense_solve": (i64, [i32, i32, P, f64, f64, i64, P, i32, P, P]),
                "orc_gs_select": (i32, [i64, i64, i32, P, P]),
                "orc_block_update": (None, [i32, i32, P, f64, f64, P, i64, i64, i32, P, i64, P, P]),
                "orc_ap_solve": (i32, [i32, i32, P, f64, f64, i64, P, i64, i32, P,
                                       i32, P, i64, i32, f64, i32, i32, i64, P, P,
                                       P, P, P, P, P, i64, P, P, P, P]),
                "orc_bcd": (i32, [i32, i32, P, f64, f64, i64, P, i64, i32, P, P, i64, P]),
                "orc_residual_rows": (None, [i32, i32, P, f64, f64, i64, P, i32, P, P, i64, P, P]),
                "orc_predict_mean": (None, [i32, i32, P, f64, f64, i64, P, P, i64, P, P]),
                "orc_grad_quadforms": (None, [i32, i32, P, f64, i64, P, i32, P, P, P, P]),
                "orc_mll_exact": (i64, [i32, i32, P, f64, f64, f64, i64, P, P, P, P]),
                "orc_mll_grad_stochastic": (i64, [i32, i32, P, f64, f64, f64, i64, P, P, i32, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    return _load().orc_num_threads()


class Hyper:
    """Kernel choice and hyperparameters (lengthscales, outputscale, noise, mean)."""

    def __init__(self, kernel: int, lengthscale, outputscale: float, noise: float, mean: float = 0.0):
        self.kernel = int(kernel)
        self.ell = _d(lengthscale).ravel()
        self.s = float(outputscale)
        self.noise = float(noise)
        self.mean = float(mean)

    @property
    def d(self) -> int:
        return self.ell.shape[0]

    @classmethod
    def of(cls, p) -> "Hyper":
        return cls(p.kernel, p.lengthscale, p.outputscale, p.noise, p.mean)


def kernel_value(h: Hyper, xi, xj) -> float:
    """s * phi(||(x - x') / l||) for one pair (Sec. 2 kernel, readings in the C header)."""
    xi, xj = _d(xi), _d(xj)
    return _load().orc_kernel_value(h.kernel, h.d, _p(h.ell), h.s, _p(xi), _p(xj))


def gram(h: Hyper, Xa, Xb=None, row0: int = 0, col0: int = 0, noise: bool = True) -> np.ndarray:
    """Dense K_hat block: s phi(x_a, x_b) + noise on the global index diagonal."""
    Xa = _d(Xa)
    Xb = Xa if Xb is None else _d(Xb)
    out = np.empty((Xa.shape[0], Xb.shape[0]))
    _load().orc_gram(h.kernel, h.d, _p(h.ell), h.s, h.noise if noise else 0.0,
                     _p(Xa), Xa.shape[0], row0, _p(Xb), Xb.shape[0], col0, _p(out))
    return out


def cholesky(A) -> np.ndarray:
    """Own Cholesky-Crout factor L (lower) of an SPD matrix; raises if not SPD."""
    L = _d(A).copy()
    bad = _load().orc_cholesky(L.shape[0], _p(L))
    if bad >= 0:
        raise np.linalg.LinAlgError(f"not SPD at pivot {bad}")
    return L


def chol_solve(L, B) -> np.ndarray:
    L = _d(L)
    B = _d(B)
    vec = B.ndim == 1
    B2 = B.reshape(B.shape[0], -1).copy()
    X = np.empty_like(B2)
    _load().orc_chol_solve(L.shape[0], _p(L), B2.shape[1], _p(B2), _p(X))
    return X.ravel() if vec else X


def dense_solve(h: Hyper, X, B) -> np.ndarray:
    """W* = K_hat^{-1} B by the dense FP64 Cholesky (the exact answer AP converges to)."""
    X = _d(X)
    B = _d(B)
    vec = B.ndim == 1
    B2 = np.ascontiguousarray(B.reshape(B.shape[0], -1))
    W = np.empty_like(B2)
    bad = _load().orc_dense_solve(h.kernel, h.d, _p(h.ell), h.s, h.noise, X.shape[0], _p(X),
                                  B2.shape[1], _p(B2), _p(W))
    if bad >= 0:
        raise np.linalg.LinAlgError(f"not SPD at pivot {bad}")
    return W.ravel() if vec else W


def gs_select(R, b: int):
    """Eq. approximate_gauss_southwell: (argmax block, all block norms ||R_J||_F^2)."""
    R = _d(R)
    R2 = np.ascontiguousarray(R.reshape(R.shape[0], -1))
    n = R2.shape[0]
    m = (n + b - 1) // b
    norms = np.empty(m)
    I = _load().orc_gs_select(n, b, R2.shape[1], _p(R2), _p(norms))
    return I, norms


def block_update(h: Hyper, X, i0: int, Delta, R, rows=None) -> np.ndarray:
    """R[rows] -= K_hat(X_rows, X_I) Delta for block I = [i0, i0 + len(Delta)) (Eq. text_update_of_r).
    Returns the updated copy of R."""
    X = _d(X)
    R = _d(R).copy()
    vec = R.ndim == 1
    R2 = R.reshape(R.shape[0], -1)
    D = np.ascontiguousarray(_d(Delta).reshape(-1, R2.shape[1]))
    rows_a = None if rows is None else np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    nrows = R2.shape[0] if rows is None else rows_a.shape[0]
    _load().orc_block_update(h.kernel, h.d, _p(h.ell), h.s, h.noise, _p(X), i0, D.shape[0],
                             R2.shape[1], _p(D), nrows, _p(rows_a), _p(R2))
    return R2.ravel() if vec else R2


class APResult:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def ap_solve(h: Hyper, X, B, b: int, select: int = SEL_GS, forced=None,
             stop: int = STOP_MEAN_REL, tol: float = 1e-6, min_epochs: int = 11,
             max_epochs: int = 1000, max_steps: int = 0, trace_cap: int = 0) -> APResult:
    """Alg. 1 (alternating projection) in FP64, step by step; see orc_ap_solve."""
    X = _d(X)
    B = _d(B)
    B2 = np.ascontiguousarray(B.reshape(B.shape[0], -1))
    n, c = B2.shape
    W = np.empty_like(B2)
    R = np.empty_like(B2)
    cap = int(trace_cap)
    trace = np.full(cap, -1, dtype=np.int32)
    energy = np.zeros(cap)
    pred = np.zeros(cap)
    chosen = np.zeros(cap)
    mx = np.zeros(cap)
    f = None if forced is None else np.ascontiguousarray(np.asarray(forced, dtype=np.int32))
    steps = ctypes.c_int64(0)
    epochs = ctypes.c_int(0)
    bad = ctypes.c_int(-1)
    rel = np.zeros(c)
    st = _load().orc_ap_solve(h.kernel, h.d, _p(h.ell), h.s, h.noise, n, _p(X), b, c, _p(B2),
                              select, _p(f), 0 if f is None else f.shape[0], stop, tol,
                              min_epochs, max_epochs, max_steps, _p(W), _p(R),
                              _p(trace), _p(energy), _p(pred), _p(chosen), _p(mx), cap,
                              ctypes.byref(steps), ctypes.byref(epochs), _p(rel), ctypes.byref(bad))
    s = steps.value
    k = min(s, cap)
    return APResult(status=st, W=W, R=R, steps=s, epochs=epochs.value, rel=rel,
                    bad_block=bad.value, trace=trace[:k], energy=energy[:k], pred_dec=pred[:k],
                    chosen_norm=chosen[:k], max_norm=mx[:k])


def bcd(h: Hyper, X, B, b: int, seq) -> np.ndarray:
    """Alg. 2 (block coordinate descent) on a given block sequence."""
    X = _d(X)
    B2 = np.ascontiguousarray(_d(B).reshape(X.shape[0], -1))
    W = np.empty_like(B2)
    seq = np.ascontiguousarray(np.asarray(seq, dtype=np.int32))
    st = _load().orc_bcd(h.kernel, h.d, _p(h.ell), h.s, h.noise, X.shape[0], _p(X), b,
                         B2.shape[1], _p(B2), _p(seq), seq.shape[0], _p(W))
    if st != OK:
        raise RuntimeError(f"orc_bcd status {st}")
    return W


def residual_rows(h: Hyper, X, B, W, rows=None) -> np.ndarray:
    """True residual rows B - K_hat W (the residual lemma of App. B), one row at a time."""
    X = _d(X)
    B2 = np.ascontiguousarray(_d(B).reshape(X.shape[0], -1))
    W2 = np.ascontiguousarray(_d(W).reshape(X.shape[0], -1))
    rows_a = None if rows is None else np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    nrows = X.shape[0] if rows is None else rows_a.shape[0]
    out = np.empty((nrows, B2.shape[1]))
    _load().orc_residual_rows(h.kernel, h.d, _p(h.ell), h.s, h.noise, X.shape[0], _p(X),
                              B2.shape[1], _p(B2), _p(W2), nrows, _p(rows_a), _p(out))
    return out


def predict_mean(h: Hyper, X, w, Xs) -> np.ndarray:
    """Posterior mean mu + K(X*, X) w (Sec. 2)."""
    X, Xs, w = _d(X), _d(Xs), _d(w).ravel()
    out = np.empty(Xs.shape[0])
    _load().orc_predict_mean(h.kernel, h.d, _p(h.ell), h.s, h.mean, X.shape[0], _p(X), _p(w),
                             Xs.shape[0], _p(Xs), _p(out))
    return out


def grad_quadforms(h: Hyper, X, U, V, alpha) -> np.ndarray:
    """sum_c alpha_c U_c^T (dK_hat/dtheta) V_c for theta = (l_1..l_d, s, sigma^2)."""
    X = _d(X)
    U = np.ascontiguousarray(_d(U).reshape(X.shape[0], -1))
    V = np.ascontiguousarray(_d(V).reshape(X.shape[0], -1))
    a = _d(alpha).ravel()
    out = np.empty(h.d + 2)
    _load().orc_grad_quadforms(h.kernel, h.d, _p(h.ell), h.s, X.shape[0], _p(X), U.shape[1],
                               _p(U), _p(V), _p(a), _p(out))
    return out


def mll_exact(h: Hyper, X, y):
    """(negative MLL without the n/2 log 2 pi constant, exact gradient over
    (l_1..l_d, s, sigma^2, mu)) by dense FP64 algebra (Eq. loss)."""
    X, y = _d(X), _d(y).ravel()
    mll = ctypes.c_double(0.0)
    grad = np.empty(h.d + 3)
    bad = _load().orc_mll_exact(h.kernel, h.d, _p(h.ell), h.s, h.noise, h.mean, X.shape[0],
                                _p(X), _p(y), ctypes.byref(mll), _p(grad))
    if bad >= 0:
        raise np.linalg.LinAlgError(f"not SPD at pivot {bad}")
    return mll.value, grad


def mll_value(h: Hyper, X, y) -> float:
    X, y = _d(X), _d(y).ravel()
    mll = ctypes.c_double(0.0)
    bad = _load().orc_mll_exact(h.kernel, h.d, _p(h.ell), h.s, h.noise, h.mean, X.shape[0],
                                _p(X), _p(y), ctypes.byref(mll), None)
    if bad >= 0:
        raise np.linalg.LinAlgError(f"not SPD at pivot {bad}")
    return mll.value


def mll_grad_stochastic(h: Hyper, X, y, Z) -> np.ndarray:
    """Eq. loss_grad_unbiased with the given probes Z (n x l), exact dense solves."""
    X, y = _d(X), _d(y).ravel()
    Z = np.ascontiguousarray(_d(Z).reshape(X.shape[0], -1))
    grad = np.empty(h.d + 3)
    bad = _load().orc_mll_grad_stochastic(h.kernel, h.d, _p(h.ell), h.s, h.noise, h.mean,
                                          X.shape[0], _p(X), _p(y), Z.shape[1], _p(Z), _p(grad))
    if bad >= 0:
        raise np.linalg.LinAlgError(f"not SPD at pivot {bad}")
    return grad
