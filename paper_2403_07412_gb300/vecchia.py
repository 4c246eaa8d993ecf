"""Python binding of the C ABI in include/vecchia.h (argument marshalling only).

Every computation runs in ``libvecchia.so``; PyTorch supplies device memory and the
current CUDA stream.  The library is loaded from this package directory and its
absence is an error: there is no CPU fallback.

The entry points keep the C names: :func:`vecchia_plan_create` (wrapped by
:class:`Plan`), :func:`vecchia_loglik`, :func:`vecchia_loglik_grad`, :func:`vecchia_loglik_range`,
:func:`vecchia_loglik_terms`, :func:`vecchia_matern`, :func:`vecchia_pivot_reciprocal`,
:func:`vecchia_mul_by_positive`,
:func:`vecchia_fp64_peak`,
:func:`vecchia_batched_prepare` and :class:`Batch` (vecchia_loglik_batched),
:func:`vecchia_loglik_noalloc`;
:class:`VecchiaLogLik` is the ``torch.autograd.Function`` over theta.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# VECCHIA_CHECKED=1 selects the bounds-checked build (build.build(checked=True))
LIB_PATH = os.path.join(HERE, "libvecchia_checked.so" if os.environ.get("VECCHIA_CHECKED", "") == "1"
                        else "libvecchia.so")

OK, EINVAL, ENOTPD, ECUDA, ETIMEOUT, ENOMEM = range(6)
ORDER_GIVEN, ORDER_RANDOM, ORDER_MAXMIN, ORDER_MORTON = 0, 1, 2, 3
KERNEL_MATERN, KERNEL_POWEXP = 0, 1
MAX_M = 150
MAX_M_WARP = 63

_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); the C ABI as declared in include/vecchia.h
SIGNATURES = {
    "vecchia_plan_create": (ctypes.c_int, [_dp, _i64, _i32, ctypes.c_int, ctypes.c_uint64,
                                           ctypes.POINTER(_i64), _vp, ctypes.POINTER(_vp)]),
    "vecchia_plan_create_sphere": (ctypes.c_int, [_dp, _i64, _i32, ctypes.c_int, ctypes.c_uint64,
                                                  ctypes.POINTER(_i64), ctypes.c_double, _vp, ctypes.POINTER(_vp)]),
    "vecchia_plan_destroy": (None, [_vp]),
    "vecchia_predict": (ctypes.c_int, [_vp, _dp, _i64, _vp, _dp, _vp, _vp, ctypes.POINTER(_i32), _vp]),
    "vecchia_plan_size": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32)]),
    "vecchia_plan_set_kernel": (ctypes.c_int, [_vp, ctypes.c_int]),
    "vecchia_covariance": (ctypes.c_int, [ctypes.c_int, _vp, _i64, _dp, _vp, _vp, _vp]),
    "vecchia_plan_perm": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "vecchia_plan_neighbors": (ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    "vecchia_loglik": (ctypes.c_int, [_vp, _vp, _dp, _vp, _vp]),
    "vecchia_loglik_grad": (ctypes.c_int, [_vp, _vp, _dp, _vp, _vp]),
    "vecchia_loglik_terms": (ctypes.c_int, [_vp, _vp, _dp, ctypes.c_int, _vp, _vp]),
    "vecchia_loglik_range": (ctypes.c_int, [_vp, _vp, _dp, _i64, _i64, ctypes.c_int, _vp, _vp]),
    "vecchia_matern": (ctypes.c_int, [_vp, _i64, _dp, _vp, _vp, _vp]),
    "vecchia_pivot_reciprocal": (ctypes.c_int, [_vp, _i64, _vp, _vp]),
    "vecchia_mul_by_positive": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "vecchia_last_error_location": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "vecchia_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "vecchia_fp64_peak": (ctypes.c_int, [_dp, _vp]),
    "vecchia_loglik_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _i32, _dp, _vp, _vp]),
    "vecchia_batched_prepare": (ctypes.c_int, [_dp, _i32, _vp]),
    "vecchia_autotune": (ctypes.c_int, [_vp, _vp, _dp, ctypes.c_int, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                        _vp]),
    "vecchia_loglik_batched": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, _vp, _i32,
                                              ctypes.c_int, _vp, _vp]),
}


class VecchiaError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().vecchia_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def lib():
    """The loaded CUDA library; raises if ``libvecchia.so`` has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_2403_07412_gb300.build.build() (nvcc, sm_103a)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(code: int, where: str) -> None:
    if code != OK:
        raise VecchiaError(code, where)


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _theta(theta) -> ctypes.Array:
    t = [float(v) for v in (theta.tolist() if hasattr(theta, "tolist") else theta)]
    if len(t) != 4:
        raise ValueError("theta must be (sigma2, beta, nu, tau2)")
    return (ctypes.c_double * 4)(*t)


def _dev_f64(x: torch.Tensor, n: int, name: str) -> torch.Tensor:
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64):
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if x.numel() != n or not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return x


class Plan:
    """Ordering and conditioning sets for one set of locations (vecchia_plan_create).

    With ``radius`` given, ``xy`` holds (longitude, latitude) in degrees and distances are
    great-circle distances on a sphere of that radius (vecchia_plan_create_sphere).
    """

    def __init__(self, xy, m: int, order: int = ORDER_RANDOM, seed: int = 0, perm=None, stream=None,
                 radius=None):
        xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
        self.n = int(xy.shape[0])
        self.m = int(m)
        self.radius = radius
        h = _vp()
        pin = None
        if order == ORDER_GIVEN:
            pin = np.ascontiguousarray(np.asarray(perm, dtype=np.int64))
        pin_p = pin.ctypes.data_as(ctypes.POINTER(_i64)) if pin is not None else None
        seed_c = ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)
        if radius is None:
            rc = lib().vecchia_plan_create(xy.ctypes.data_as(_dp), self.n, self.m, int(order), seed_c, pin_p,
                                           _vp(_stream(stream)), ctypes.byref(h))
            _check(rc, "vecchia_plan_create")
        else:
            rc = lib().vecchia_plan_create_sphere(xy.ctypes.data_as(_dp), self.n, self.m, int(order), seed_c,
                                                  pin_p, float(radius), _vp(_stream(stream)), ctypes.byref(h))
            _check(rc, "vecchia_plan_create_sphere")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().vecchia_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_kernel(self, kernel: int) -> None:
        """Covariance family of this plan's likelihood calls (KERNEL_MATERN or KERNEL_POWEXP)."""
        _check(lib().vecchia_plan_set_kernel(self._h, int(kernel)), "vecchia_plan_set_kernel")

    def perm(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int64)
        _check(lib().vecchia_plan_perm(self._h, out.ctypes.data_as(ctypes.POINTER(_i64))), "vecchia_plan_perm")
        return out

    def neighbors(self) -> np.ndarray:
        out = np.empty((self.n, self.m), dtype=np.int32)
        _check(lib().vecchia_plan_neighbors(self._h, out.ctypes.data_as(ctypes.POINTER(_i32))),
               "vecchia_plan_neighbors")
        return out

    def last_error_location(self) -> int:
        loc = _i64(-1)
        lib().vecchia_last_error_location(self._h, ctypes.byref(loc))
        return int(loc.value)

    def last_error(self):
        """(first failing ordered location or -1, status): ENOTPD for a block that is not
        positive definite, EINVAL for non-finite data, OK for none."""
        loc = _i64(-1)
        rc = lib().vecchia_last_error_location(self._h, ctypes.byref(loc))
        return int(loc.value), int(rc)


def vecchia_loglik(plan: Plan, y: torch.Tensor, theta, out: torch.Tensor | None = None, stream=None):
    y = _dev_f64(y, plan.n, "y")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=y.device)
    rc = lib().vecchia_loglik(plan.handle, _vp(y.data_ptr()), _theta(theta), _vp(out.data_ptr()),
                              _vp(_stream(stream)))
    _check(rc, "vecchia_loglik")
    return out


def vecchia_loglik_grad(plan: Plan, y: torch.Tensor, theta, out: torch.Tensor | None = None, stream=None):
    y = _dev_f64(y, plan.n, "y")
    if out is None:
        out = torch.empty(4, dtype=torch.float64, device=y.device)
    rc = lib().vecchia_loglik_grad(plan.handle, _vp(y.data_ptr()), _theta(theta), _vp(out.data_ptr()),
                                   _vp(_stream(stream)))
    _check(rc, "vecchia_loglik_grad")
    return out


def vecchia_loglik_range(plan: Plan, y: torch.Tensor, theta, i0: int, i1: int, want_grad: bool = False,
                         out: torch.Tensor | None = None, stream=None):
    """The contribution of ordered locations [i0, i1) to l (and its gradient if want_grad)."""
    y = _dev_f64(y, plan.n, "y")
    if out is None:
        out = torch.empty(4 if want_grad else 1, dtype=torch.float64, device=y.device)
    rc = lib().vecchia_loglik_range(plan.handle, _vp(y.data_ptr()), _theta(theta), int(i0), int(i1),
                                    1 if want_grad else 0, _vp(out.data_ptr()), _vp(_stream(stream)))
    _check(rc, "vecchia_loglik_range")
    return out


def vecchia_loglik_terms(plan: Plan, y: torch.Tensor, theta, want_grad: bool = False,
                         out: torch.Tensor | None = None, stream=None):
    y = _dev_f64(y, plan.n, "y")
    w = 4 if want_grad else 1
    if out is None:
        out = torch.empty((plan.n, w), dtype=torch.float64, device=y.device)
    rc = lib().vecchia_loglik_terms(plan.handle, _vp(y.data_ptr()), _theta(theta), 1 if want_grad else 0,
                                    _vp(out.data_ptr()), _vp(_stream(stream)))
    _check(rc, "vecchia_loglik_terms")
    return out if want_grad else out[:, 0]


def vecchia_matern(d: torch.Tensor, theta, with_dbeta: bool = True, stream=None):
    d = _dev_f64(d, d.numel(), "d")
    c = torch.empty_like(d)
    dc = torch.empty_like(d) if with_dbeta else None
    rc = lib().vecchia_matern(_vp(d.data_ptr()), d.numel(), _theta(theta), _vp(c.data_ptr()),
                              _vp(dc.data_ptr()) if dc is not None else None, _vp(_stream(stream)))
    _check(rc, "vecchia_matern")
    return (c, dc) if with_dbeta else c


def vecchia_pivot_reciprocal(d: torch.Tensor, stream=None) -> torch.Tensor:
    """The LDL^T pivot reciprocal of the likelihood kernels: 1/d, NaN outside [2^-1022, 2^1022)."""
    d = _dev_f64(d, d.numel(), "d")
    out = torch.empty_like(d)
    rc = lib().vecchia_pivot_reciprocal(_vp(d.data_ptr()), d.numel(), _vp(out.data_ptr()), _vp(_stream(stream)))
    _check(rc, "vecchia_pivot_reciprocal")
    return out


def vecchia_mul_by_positive(a: torch.Tensor, b: torch.Tensor, stream=None) -> torch.Tensor:
    """The kernels' integer column-scaling product a * b (b a positive normal double)."""
    a = _dev_f64(a, a.numel(), "a")
    b = _dev_f64(b, a.numel(), "b")
    out = torch.empty_like(a)
    rc = lib().vecchia_mul_by_positive(_vp(a.data_ptr()), _vp(b.data_ptr()), a.numel(), _vp(out.data_ptr()),
                                       _vp(_stream(stream)))
    _check(rc, "vecchia_mul_by_positive")
    return out


def vecchia_loglik_noalloc(xy: torch.Tensor, y: torch.Tensor, nbr: torch.Tensor, self_idx: torch.Tensor,
                           m: int, theta, out: torch.Tensor, stream=None):
    """Allocation-free log-likelihood over caller-owned device arrays (see the C header):
    xy (n x 2, original order), y (n), nbr (n x m int32 original indices of each ordered
    location's conditioning set, -1 padded), self_idx (n int32, perm).  Writes out[0]."""
    n = y.numel()
    for t, name, dt, cnt in ((xy, "xy", torch.float64, 2 * n), (y, "y", torch.float64, n),
                             (nbr, "nbr", torch.int32, n * m), (self_idx, "self_idx", torch.int32, n),
                             (out, "out", torch.float64, None)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous CUDA {dt} tensor")
        if cnt is not None and t.numel() != cnt:
            raise ValueError(f"{name} must have {cnt} elements")
    rc = lib().vecchia_loglik_noalloc(_vp(xy.data_ptr()), _vp(y.data_ptr()), _vp(nbr.data_ptr()),
                                      _vp(self_idx.data_ptr()), n, int(m), _theta(theta), _vp(out.data_ptr()),
                                      _vp(_stream(stream)))
    _check(rc, "vecchia_loglik_noalloc")
    return out


def vecchia_autotune(plan: Plan, y: torch.Tensor, theta, want_grad: bool = True, stream=None):
    """Time the launch shapes for this plan's block size; returns (lanes per location, warps per CTA)."""
    y = _dev_f64(y, plan.n, "y")
    g, w = _i32(0), _i32(0)
    _check(lib().vecchia_autotune(plan.handle, _vp(y.data_ptr()), _theta(theta), 1 if want_grad else 0,
                                  ctypes.byref(g), ctypes.byref(w), _vp(_stream(stream))), "vecchia_autotune")
    return int(g.value), int(w.value)


def vecchia_batched_prepare(nus, stream=None) -> None:
    """Prepare the covariance tables (one per smoothness value) for the batched call."""
    arr = (ctypes.c_double * len(nus))(*[float(v) for v in nus])
    _check(lib().vecchia_batched_prepare(arr, len(nus), _vp(_stream(stream))), "vecchia_batched_prepare")


class Batch:
    """Argument bundle for vecchia_loglik_batched over fixed plans and field arrays."""

    def __init__(self, plans, ys, ntheta: int, want_grad: bool = True):
        if len(plans) != len(ys):
            raise ValueError("one field array per plan")
        self.plans = list(plans)
        self.ys = [_dev_f64(y, p.n, "y") for p, y in zip(plans, ys)]
        self.ntheta = int(ntheta)
        self.want_grad = bool(want_grad)
        self._ph = (_vp * len(plans))(*[p.handle.value for p in plans])
        self._yh = (_vp * len(plans))(*[y.data_ptr() for y in self.ys])

    def run(self, thetas: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        nf = len(self.plans)
        w = 4 if self.want_grad else 1
        if not (thetas.is_cuda and thetas.dtype == torch.float64 and thetas.is_contiguous()
                and thetas.numel() == nf * self.ntheta * 4):
            raise ValueError("thetas must be a contiguous CUDA float64 tensor of shape (nfields, ntheta, 4)")
        if out is None:
            out = torch.empty((nf, self.ntheta, w), dtype=torch.float64, device=thetas.device)
        rc = lib().vecchia_loglik_batched(self._ph, self._yh, nf, _vp(thetas.data_ptr()), self.ntheta,
                                          1 if self.want_grad else 0, _vp(out.data_ptr()), _vp(_stream(stream)))
        _check(rc, "vecchia_loglik_batched")
        return out


def vecchia_predict(plan: Plan, xy_new, y, theta, with_var: bool = True, return_neighbors: bool = False,
                    stream=None):
    """Kriging at new locations from the m nearest observed points of ``plan``:
    (mean, var) as CUDA float64 tensors (var None unless ``with_var``), plus the
    conditioning sets (n_new x m original indices) when ``return_neighbors``."""
    xn = np.ascontiguousarray(np.asarray(xy_new, dtype=np.float64).reshape(-1, 2))
    k = int(xn.shape[0])
    y = _dev_f64(y, plan.n, "y")
    mean = torch.empty(k, dtype=torch.float64, device=y.device)
    var = torch.empty(k, dtype=torch.float64, device=y.device) if with_var else None
    nbr = np.empty((k, plan.m), dtype=np.int32) if return_neighbors else None
    rc = lib().vecchia_predict(plan.handle, xn.ctypes.data_as(_dp), k, _vp(y.data_ptr()), _theta(theta),
                               _vp(mean.data_ptr()), _vp(var.data_ptr()) if var is not None else None,
                               nbr.ctypes.data_as(ctypes.POINTER(_i32)) if nbr is not None else None,
                               _vp(_stream(stream)))
    _check(rc, "vecchia_predict")
    return (mean, var, nbr) if return_neighbors else (mean, var)


def vecchia_covariance(kernel: int, d: torch.Tensor, theta, with_dbeta: bool = True, stream=None):
    """C(d) (and dC/dbeta) of either covariance family through the kernels' device code."""
    d = _dev_f64(d, d.numel(), "d")
    c = torch.empty_like(d)
    dc = torch.empty_like(d) if with_dbeta else None
    rc = lib().vecchia_covariance(int(kernel), _vp(d.data_ptr()), d.numel(), _theta(theta), _vp(c.data_ptr()),
                                  _vp(dc.data_ptr()) if dc is not None else None, _vp(_stream(stream)))
    _check(rc, "vecchia_covariance")
    return (c, dc) if with_dbeta else c


def vecchia_fp64_peak(stream=None) -> float:
    g = ctypes.c_double(0.0)
    _check(lib().vecchia_fp64_peak(ctypes.byref(g), _vp(_stream(stream))), "vecchia_fp64_peak")
    return float(g.value)


class VecchiaLogLik(torch.autograd.Function):
    """l(theta) as a differentiable function of theta = (sigma2, beta, nu, tau2).

    Backward uses the library's adjoint for (sigma2, beta, tau2) and a central finite
    difference of the forward kernel for nu (step ``nu_step`` relative).
    """

    @staticmethod
    def forward(ctx, theta: torch.Tensor, plan: Plan, y: torch.Tensor, nu_step: float = 1e-6):
        th = theta.detach().to("cpu", torch.float64)
        g = vecchia_loglik_grad(plan, y, th)
        ctx.plan, ctx.y, ctx.nu_step = plan, y, nu_step
        ctx.save_for_backward(theta.detach())
        ctx.g = g
        return g[0:1].clone().reshape(()).to(theta.device)

    @staticmethod
    def backward(ctx, gout):
        (theta,) = ctx.saved_tensors
        th = theta.to("cpu", torch.float64)
        nu = float(th[2])
        h = ctx.nu_step * nu
        tp, tm = th.clone(), th.clone()
        tp[2] = nu + h
        tm[2] = nu - h
        lp = vecchia_loglik(ctx.plan, ctx.y, tp)
        lm = vecchia_loglik(ctx.plan, ctx.y, tm)
        dnu = (lp - lm) / (2.0 * h)
        g = ctx.g
        grad = torch.stack([g[1], g[2], dnu[0], g[3]]).to(theta.device, theta.dtype)
        return gout * grad, None, None, None
