"""GB300 alternating-projection solver for Gaussian-process kernel systems.

Python binding of libap.so (include/ap.h).  The functions keep the C names and
only marshal arguments: tensors must be CUDA float32 and contiguous, their
device pointers go straight to the library, and every step of the solver runs
in the library's CUDA kernels.  There is no CPU fallback: if libap.so cannot be
built or loaded, importing the binding raises.

Method: Wu et al., "Large-Scale Gaussian Processes via Alternating
Projection" (AISTATS 2024), Alg. 1 with the modified Gauss-Southwell rule and
cached block Cholesky factors.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional, Sequence

import numpy as np

from . import _capi
from ._capi import (AP_ERR_SCRATCH_LIMIT, AP_ERR_CANCELLED, AP_BF16_REFINE, AP_ERR_CUDA, AP_ERR_INVALID_ARG, AP_ERR_NAN, AP_ERR_NOMEM,  # noqa: F401
                    AP_ERR_NOT_CONVERGED, AP_ERR_NOT_SPD, AP_ERR_TIMEOUT, AP_ERR_UNSUPPORTED,
                    AP_FP16_REFINE, AP_FP32, AP_MATERN32, AP_MATERN52, AP_OK, AP_RBF, AP_SEL_CYCLIC,
                    AP_SEL_GS, AP_SEL_RANDOM, AP_STOP_FRO, AP_STOP_MAX_REL, AP_STOP_MEAN_REL,
                    AP_STOP_Y_REL, AP_RESID_AUTO, AP_RESID_FP32, AP_RESID_COMPENSATED, AP_CACHE_TC_EXACT,
                    AP_CACHE_FP64)

__all__ = ["ApError", "Hyper", "Context", "ap_opts_default", "ap_create", "ap_set_hyper", "ap_solve",
           "ap_residual", "ap_predict_mean", "ap_grad_quadforms", "ap_mll_grad", "ap_destroy",
           "ap_status_str", "ap_launch_count", "ap_sfu_rates", "ap_phi_fp64_eval", "ap_grad_quadforms_static", "ap_tracked_residual", "ap_device_bytes", "ap_solve_host", "ap_bounds_violations", "ap_bounds_selftest", "ApServer",
           "MLLDataFit"]


class ApError(RuntimeError):
    def __init__(self, status: int, where: str, ctx=None):
        msg = f"{where}: {ap_status_str(status)}"
        self.cuda_error = 0
        if ctx is not None and status == AP_ERR_CUDA:
            self.cuda_error = int(_capi.load().ap_last_cuda_error(ctx.handle))
            msg += f" (cudaError_t {self.cuda_error})"
        super().__init__(msg)
        self.status = status


def _torch():
    import torch
    return torch


def ap_status_str(status: int) -> str:
    return _capi.load().ap_status_str(int(status)).decode()


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float32 tensor")
    return t.data_ptr()


@dataclasses.dataclass
class Hyper:
    """Kernel family and hyperparameters (lengthscales, outputscale, noise, mean)."""
    kernel: int
    lengthscale: Sequence[float]
    outputscale: float = 1.0
    noise: float = 0.1
    mean: float = 0.0

    def to_c(self):
        ell = np.ascontiguousarray(np.asarray(self.lengthscale, dtype=np.float32).ravel())
        h = _capi.ap_hyper(int(self.kernel), int(ell.shape[0]), ell.ctypes.data, float(self.outputscale),
                           float(self.noise), float(self.mean))
        return h, ell  # keep ell alive while h is used


def ap_opts_default(**overrides) -> _capi.ap_opts:
    o = _capi.ap_opts()
    _capi.load().ap_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class Context:
    """Owner of an ap_ctx* plus the objects whose memory it borrows."""

    def __init__(self, handle, X, n: int, d: int, opts):
        self.handle = handle
        self.X = X
        self.n = n
        self.d = d
        self.opts = opts
        self._trace = None

    def __del__(self):
        try:
            ap_destroy(self)
        except Exception:
            pass


def ap_create(X, hyper: Hyper, opts: Optional[_capi.ap_opts] = None, trace_cap: int = 0) -> Context:
    """Build a context (and the FP64 Cholesky cache) for the n x d inputs X."""
    torch = _torch()
    L = _capi.load()
    opts = opts or ap_opts_default()
    if opts.stream is None or opts.stream == 0:
        opts.stream = torch.cuda.current_stream(X.device).cuda_stream
    trace = None
    if trace_cap > 0:
        trace = (ctypes.c_int32 * trace_cap)()
        opts.block_trace = ctypes.cast(trace, ctypes.POINTER(ctypes.c_int32))
        opts.trace_cap = trace_cap
    h, ell = hyper.to_c()
    handle = ctypes.c_void_p()
    st = L.ap_create(ctypes.byref(handle), _ptr(X), X.shape[0], X.shape[1], ctypes.byref(h), ctypes.byref(opts))
    if st != AP_OK:
        raise ApError(st, "ap_create")
    ctx = Context(handle, X, X.shape[0], X.shape[1], opts)
    ctx._trace = trace
    return ctx


def ap_set_hyper(ctx: Context, hyper: Hyper) -> None:
    h, ell = hyper.to_c()
    st = _capi.load().ap_set_hyper(ctx.handle, ctypes.byref(h))
    if st != AP_OK:
        raise ApError(st, "ap_set_hyper", ctx)


def info_dict(info: _capi.ap_info) -> dict:
    c = info.c
    return dict(epochs=info.epochs, steps=info.steps, refinements=info.refinements, bad_block=info.bad_block,
                c=c, rel_res_tracked=list(info.rel_res_tracked[:c]), rel_res_true=list(info.rel_res_true[:c]),
                t_cache_s=info.t_cache_s, t_solve_s=info.t_solve_s, t_refine_s=info.t_refine_s,
                kernel_entries=info.kernel_entries, entries_per_s=info.entries_per_s,
                gpu_launches=info.gpu_launches, data_fit=info.data_fit, t_update_s=info.t_update_s,
                n_update=info.n_update, t_blocksolve_s=info.t_blocksolve_s, fp32_epochs=info.fp32_epochs,
                compensated=bool(info.compensated), diverged=int(info.diverged))


def ap_solve(ctx: Context, B, W0=None, W=None):
    """Solve K_hat W = B (Alg. 1).  Returns (status, W, info dict, block trace)."""
    torch = _torch()
    B2 = B if B.dim() == 2 else B.reshape(-1, 1)
    c = B2.shape[1]
    if W is None:
        W = torch.empty_like(B2)
    info = _capi.ap_info()
    st = _capi.load().ap_solve(ctx.handle, _ptr(B2), c, _ptr(W0), _ptr(W), ctypes.byref(info))
    if st not in (AP_OK, AP_ERR_NOT_CONVERGED):
        raise ApError(st, "ap_solve", ctx)
    trace = None
    if ctx._trace is not None:
        trace = np.frombuffer(ctx._trace, dtype=np.int32)[:min(info.steps, ctx.opts.trace_cap)].copy()
    return st, W, info_dict(info), trace


def ap_solve_host(X: np.ndarray, B: np.ndarray, hyper: Hyper, opts=None, W: Optional[np.ndarray] = None):
    """One-shot solve for host arrays (float32, C-contiguous; page-locked memory
    such as a pinned torch tensor's numpy view copies fastest): copies in,
    builds the cache, runs Alg. 1, copies W out.  Returns (status, W, info)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    B2 = np.ascontiguousarray(B, dtype=np.float32).reshape(X.shape[0], -1)
    if W is None:
        W = np.empty_like(B2)
    opts = opts or ap_opts_default()
    h, ell = hyper.to_c()
    info = _capi.ap_info()
    st = _capi.load().ap_solve_host(X.ctypes.data, X.shape[0], X.shape[1], ctypes.byref(h), ctypes.byref(opts),
                                    B2.ctypes.data, B2.shape[1], W.ctypes.data, ctypes.byref(info))
    if st not in (AP_OK, AP_ERR_NOT_CONVERGED):
        raise ApError(st, "ap_solve_host")
    return st, W, info_dict(info)


def ap_residual(ctx: Context, B, W, R=None):
    """R = B - K_hat W in the FP32 form, all n^2 entries on the fly."""
    torch = _torch()
    B2 = B if B.dim() == 2 else B.reshape(-1, 1)
    W2 = W if W.dim() == 2 else W.reshape(-1, 1)
    if R is None:
        R = torch.empty_like(B2)
    st = _capi.load().ap_residual(ctx.handle, _ptr(B2), B2.shape[1], _ptr(W2), _ptr(R))
    if st != AP_OK:
        raise ApError(st, "ap_residual", ctx)
    return R


def ap_predict_mean(ctx: Context, w, Xs, out=None):
    """mu + K(X*, X) w for the test inputs Xs (M x d)."""
    torch = _torch()
    if out is None:
        out = torch.empty(Xs.shape[0], device=Xs.device, dtype=torch.float32)
    st = _capi.load().ap_predict_mean(ctx.handle, _ptr(w), _ptr(Xs), Xs.shape[0], _ptr(out))
    if st != AP_OK:
        raise ApError(st, "ap_predict_mean", ctx)
    return out


def ap_grad_quadforms(ctx: Context, U, V, alpha) -> np.ndarray:
    """sum_c alpha_c U_c^T dK_hat/dtheta V_c for theta = (l_1..l_d, s, sigma^2)."""
    U2 = U if U.dim() == 2 else U.reshape(-1, 1)
    V2 = V if V.dim() == 2 else V.reshape(-1, 1)
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
    out = np.zeros(ctx.d + 2)
    st = _capi.load().ap_grad_quadforms(ctx.handle, _ptr(U2), _ptr(V2), U2.shape[1], a.ctypes.data,
                                        out.ctypes.data)
    if st != AP_OK:
        raise ApError(st, "ap_grad_quadforms", ctx)
    return out


def ap_grad_quadforms_static(ctx: Context, U, V, alpha) -> np.ndarray:
    """ap_grad_quadforms without device allocation (fixed scratch inside libap.so),
    for callers that may not allocate once their steady state has begun (serving
    loops, processes whose own pool holds the free HBM).  c must be 1, 4, 16 or
    32; overlapping calls share the scratch and must be serialised."""
    U2 = U if U.dim() == 2 else U.reshape(-1, 1)
    V2 = V if V.dim() == 2 else V.reshape(-1, 1)
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
    out = np.zeros(ctx.d + 2)
    st = _capi.load().ap_grad_quadforms_static(ctx.handle, _ptr(U2), _ptr(V2), U2.shape[1], a.ctypes.data,
                                               out.ctypes.data)
    if st != AP_OK:
        raise ApError(st, "ap_grad_quadforms_static", ctx)
    return out


def ap_mll_grad(ctx: Context, y, n_probes: int, Z=None):
    """Stochastic MLL gradient (Eq. loss_grad_unbiased) over (l_1..l_d, s, sigma^2, mu).
    Returns (status, grad as float32 numpy array, info dict)."""
    g = np.zeros(ctx.d + 3, dtype=np.float32)
    info = _capi.ap_info()
    st = _capi.load().ap_mll_grad(ctx.handle, _ptr(y), int(n_probes), _ptr(Z), g.ctypes.data, ctypes.byref(info))
    if st not in (AP_OK, AP_ERR_NOT_CONVERGED):
        raise ApError(st, "ap_mll_grad", ctx)
    return st, g, info_dict(info)


def ap_launch_count(ctx: Context) -> int:
    return int(_capi.load().ap_launch_count(ctx.handle))


def ap_bounds_violations():
    """(count, "unit:line" of the first) of failed index checks since the last
    call, in the bounds-checked build (AP_CHECKED=1); (-1, "") in the product
    build.  Synchronises the device."""
    buf = ctypes.create_string_buffer(256)
    n = int(_capi.load().ap_bounds_violations(buf, 256))
    return n, buf.value.decode()


def ap_bounds_selftest(index: int) -> int:
    """Status of a one-thread read of element `index` of an 8-element buffer
    through the index check (recorded when out of range, checked build only)."""
    return int(_capi.load().ap_bounds_selftest(int(index)))


def ap_device_bytes(ctx: Context) -> int:
    """Device bytes the context holds right now."""
    return int(_capi.load().ap_device_bytes(ctx.handle))


def ap_tracked_residual(ctx: Context, c: int, R=None):
    """The residual the last solve tracked (n x c), for verification."""
    torch = _torch()
    if R is None:
        R = torch.empty((ctx.n, c), dtype=torch.float32, device=ctx.X.device)
    st = _capi.load().ap_tracked_residual(ctx.handle, c, _ptr(R))
    if st != AP_OK:
        raise ApError(st, "ap_tracked_residual", ctx)
    return R


def ap_sfu_rates() -> tuple:
    """(exp2, sqrt) SFU results per SM clock, measured on the current device."""
    e, q = ctypes.c_double(), ctypes.c_double()
    st = _capi.load().ap_sfu_rates(ctypes.byref(e), ctypes.byref(q))
    if st != AP_OK:
        raise ApError(st, "ap_sfu_rates")
    return e.value, q.value


def ap_phi_fp64_eval(kernel: int, r2) -> np.ndarray:
    """FP64 phi(r^2) as the Cholesky cache evaluates it on the device."""
    r2 = np.ascontiguousarray(r2, dtype=np.float64).ravel()
    out = np.empty_like(r2)
    st = _capi.load().ap_phi_fp64_eval(int(kernel), r2.ctypes.data_as(ctypes.c_void_p), r2.size,
                                       out.ctypes.data_as(ctypes.c_void_p))
    if st != AP_OK:
        raise ApError(st, "ap_phi_fp64_eval")
    return out


def ap_destroy(ctx: Context) -> None:
    if ctx is not None and ctx.handle:
        _capi.load().ap_destroy(ctx.handle)
        ctx.handle = None


class ApServer:
    """Continuous-batching server (ap_server_*): GP solve + posterior mean per
    request, admitted by HBM budget, overlapping on the device.  Keeps the
    host arrays of every request alive until the server is closed."""

    def __init__(self, hbm_budget: int, slots: int = 4, device: int = 0):
        self.L = _capi.load()
        self.handle = ctypes.c_void_p()
        st = self.L.ap_server_create(ctypes.byref(self.handle), int(hbm_budget), int(slots), int(device))
        if st != AP_OK:
            raise ApError(st, "ap_server_create")
        self._keep = {}

    def submit(self, X, y, Xtest, hyper: Hyper, block: int = 4096, tol: float = 1e-2,
               stop: int = AP_STOP_MAX_REL, min_epochs: int = 1, max_epochs: int = 1000,
               precision: int = AP_FP32, refine_every: int = 4) -> int:
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32).ravel()
        Xt = np.ascontiguousarray(Xtest, dtype=np.float32)
        mean = np.zeros(Xt.shape[0], dtype=np.float32)
        h, ell = hyper.to_c()
        r = _capi.ap_request(X.ctypes.data, X.shape[0], X.shape[1], y.ctypes.data, Xt.ctypes.data, Xt.shape[0],
                             h, int(block), float(tol), int(stop), int(min_epochs), int(max_epochs),
                             int(precision), int(refine_every), mean.ctypes.data)
        rid = ctypes.c_int64(0)
        st = self.L.ap_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid))
        if st != AP_OK:
            raise ApError(st, "ap_server_submit")
        self._keep[rid.value] = (X, y, Xt, mean, ell)
        return rid.value

    @staticmethod
    def _res(res) -> dict:
        return dict(done=bool(res.done), status=res.status, epochs=res.epochs, rel_res=res.rel_res,
                    queue_s=res.queue_s, latency_s=res.latency_s, reserved_bytes=res.reserved_bytes,
                    started=bool(res.started), compensated=bool(res.compensated))

    def cancel(self, rid: int) -> None:
        """Drop a queued request, or stop a running one at the end of its epoch."""
        st = self.L.ap_server_cancel(self.handle, int(rid))
        if st != AP_OK:
            raise ApError(st, "ap_server_cancel")

    def poll(self, rid: int) -> dict:
        res = _capi.ap_request_result()
        st = self.L.ap_server_poll(self.handle, int(rid), ctypes.byref(res))
        if st != AP_OK:
            raise ApError(st, "ap_server_poll")
        return self._res(res)

    def wait(self, rid: int, timeout_s: float = 600.0) -> dict:
        res = _capi.ap_request_result()
        st = self.L.ap_server_wait(self.handle, int(rid), float(timeout_s), ctypes.byref(res))
        if st != AP_OK:
            raise ApError(st, "ap_server_wait")
        return self._res(res)

    def mean(self, rid: int) -> np.ndarray:
        return self._keep[rid][3]

    def close(self) -> None:
        if self.handle:
            self.L.ap_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLLDataFit:
    """torch.autograd.Function wrapper: forward returns the data-fit term
    1/2 (y - mu)^T K_hat^{-1} (y - mu); backward returns the stochastic gradient
    of the full negative MLL (Eq. loss_grad_unbiased) with respect to
    (lengthscale, outputscale, noise, mean).  AP yields no log-determinant, so
    the forward value is not the MLL itself (the paper's Sec. 6 limitation)."""

    @staticmethod
    def apply(ctx: Context, y, kernel: int, lengthscale, outputscale, noise, mean, n_probes: int = 15, Z=None):
        torch = _torch()

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(fctx, ell, s, sig2, mu):
                hyper = Hyper(kernel, ell.detach().cpu().numpy(), float(s), float(sig2), float(mu))
                ap_set_hyper(ctx, hyper)
                _, g, info = ap_mll_grad(ctx, y, n_probes, Z)
                fctx.save_for_backward(torch.from_numpy(g.astype(np.float64)))
                fctx.d = ell.numel()
                return torch.tensor(info["data_fit"], dtype=torch.float64)

            @staticmethod
            def backward(fctx, go):
                (g,) = fctx.saved_tensors
                d = fctx.d
                go = go.detach().cpu().double()
                return (go * g[:d], go * g[d], go * g[d + 1], go * g[d + 2])

        return _Fn.apply(lengthscale, outputscale, noise, mean)
