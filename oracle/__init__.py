"""Vecchia log-likelihood ORACLE — test infrastructure, not part of the product.

A plain, slow FP64 CPU implementation of the Vecchia-approximated Gaussian
log-likelihood (arXiv 2403.07412), written from the paper and sharing no code
with the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.

What each function follows:

* :func:`matern` — Eq. (2) (Sec. IV-A), through ``std::cyl_bessel_k``;
  :func:`powexp` — Eq. (3), the power-exponential family of the real-data model.
* :func:`loglik_exact` — Eq. (1), dense, with the oracle's own Cholesky.
* :func:`order_random` / :func:`order_maxmin` (and its prefix,
  :func:`order_maxmin_prefix`) / :func:`order_morton` — Sec. V-A
  orderings (random = splitmix64-driven Fisher–Yates; maxmin = greedy farthest
  point from the point nearest the centroid, ties to the lowest index; Morton =
  Z-order of 16-bit cell indices).
* :func:`knn_rows` — Algorithm 1, nearest-neighbour loop: the m nearest
  *previously ordered* points, ties by index, brute force; :func:`knn_rows_sphere`
  the same on the sphere (keys: squared chord of unit vectors).
* :func:`predict` — kriging at new locations from the m nearest observed ones (the
  paper's prediction experiment, Sec. VI-C / Table III), by the Vecchia conditional
  mean and variance.
* :func:`gcd` — Sec. VI-C great-circle distance (haversine); ``radius=`` switches
  :func:`vecchia_rows` / :func:`loglik_exact` to it for (longitude, latitude) data.
* :func:`vecchia_rows` / :func:`vecchia` — Sec. V-B: the Vecchia product of
  univariate conditionals, explicit conditional mean and variance, and the
  gradient in (sigma^2, beta, tau^2) by the joint-minus-marginal trace identity.

Every function here is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vecchia_oracle.cpp")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle's C++ source into ``oracle/_liboracle.so``."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c_int, c_i64, c_i32, c_d, c_u64 = (ctypes.c_int, ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_double, ctypes.c_uint64)
        sig = {
            "oracle_num_threads": (c_int, []),
            "oracle_set_threads": (None, [c_int]),
            "oracle_matern": (c_int, [c_i64, _dp, c_d, c_d, c_d, _dp]),
            "oracle_matern_dbeta": (c_int, [c_i64, _dp, c_d, c_d, c_d, _dp]),
            "oracle_bessel_k": (c_int, [c_i64, _dp, c_d, _dp]),
            "oracle_powexp": (c_int, [c_i64, _dp, c_d, c_d, c_d, _dp]),
            "oracle_powexp_dbeta": (c_int, [c_i64, _dp, c_d, c_d, c_d, _dp]),
            "oracle_splitmix64": (None, [c_u64, c_i64, _u64p]),
            "oracle_order_random": (c_int, [c_i64, c_u64, _i64p]),
            "oracle_order_maxmin": (c_int, [c_i64, _dp, _i64p]),
            "oracle_order_maxmin_prefix": (c_int, [c_i64, _dp, c_i64, _i64p]),
            "oracle_order_morton": (c_int, [c_i64, _dp, _i64p]),
            "oracle_knn_rows": (c_int, [c_i64, _dp, c_i32, _i64p, c_i64, _i32p]),
            "oracle_vecchia_rows": (c_int, [c_i64, _dp, _dp, c_i32, _dp, _i64p, c_i64, _i32p, c_int,
                                            _dp, _dp, _i64p, c_int, c_int, c_d]),
            "oracle_sphere_xyz": (None, [c_i64, _dp, _dp]),
            "oracle_gcd": (None, [c_i64, _dp, _dp, c_d, _dp]),
            "oracle_knn_rows_sphere": (c_int, [c_i64, _dp, c_i32, _i64p, c_i64, _i32p]),
            "oracle_predict": (c_int, [c_i64, _dp, _dp, c_i64, _dp, c_i32, _dp, c_int, c_int, c_d, _dp, _dp,
                                       _i32p]),
            "oracle_sum_columns": (None, [c_i64, c_i32, _dp, _dp]),
            "oracle_loglik_exact": (c_int, [c_i64, _dp, _dp, _dp, _dp, _dp, c_int, c_int, c_d]),
            "oracle_block_logdensity": (c_int, [c_i32, _dp, _dp, _dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def matern(d, sigma2: float, beta: float, nu: float) -> np.ndarray:
    """Eq. (2) covariance at distances ``d`` (C(0) = sigma2)."""
    d = _f64(np.atleast_1d(d))
    out = np.empty_like(d)
    _load().oracle_matern(d.size, _p(d, _dp), sigma2, beta, nu, _p(out, _dp))
    return out


def matern_dbeta(d, sigma2: float, beta: float, nu: float) -> np.ndarray:
    """dC/dbeta of Eq. (2) at distances ``d``."""
    d = _f64(np.atleast_1d(d))
    out = np.empty_like(d)
    _load().oracle_matern_dbeta(d.size, _p(d, _dp), sigma2, beta, nu, _p(out, _dp))
    return out


def powexp(d, sigma2: float, beta: float, alpha: float) -> np.ndarray:
    """Eq. (3) covariance sigma2 exp(-d^alpha / beta) at distances ``d``."""
    d = _f64(np.atleast_1d(d))
    out = np.empty_like(d)
    _load().oracle_powexp(d.size, _p(d, _dp), sigma2, beta, alpha, _p(out, _dp))
    return out


def powexp_dbeta(d, sigma2: float, beta: float, alpha: float) -> np.ndarray:
    """dC/dbeta of Eq. (3)."""
    d = _f64(np.atleast_1d(d))
    out = np.empty_like(d)
    _load().oracle_powexp_dbeta(d.size, _p(d, _dp), sigma2, beta, alpha, _p(out, _dp))
    return out


def bessel_k(x, nu: float) -> np.ndarray:
    """K_nu(x) as the oracle evaluates it (``std::cyl_bessel_k``)."""
    x = _f64(np.atleast_1d(x))
    out = np.empty_like(x)
    _load().oracle_bessel_k(x.size, _p(x, _dp), nu, _p(out, _dp))
    return out


def splitmix64(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().oracle_splitmix64(ctypes.c_uint64(seed), count, _p(out, _u64p))
    return out


def order_random(n: int, seed: int) -> np.ndarray:
    """Random ordering: perm[k] = original index of the k-th ordered location."""
    perm = np.empty(n, dtype=np.int64)
    _load().oracle_order_random(n, ctypes.c_uint64(seed), _p(perm, _i64p))
    return perm


def order_maxmin(xy) -> np.ndarray:
    """Exact maxmin ordering, O(n^2)."""
    xy = _f64(xy).reshape(-1, 2)
    perm = np.empty(xy.shape[0], dtype=np.int64)
    _load().oracle_order_maxmin(xy.shape[0], _p(xy, _dp), _p(perm, _i64p))
    return perm


def order_maxmin_prefix(xy, count: int) -> np.ndarray:
    """The first ``count`` entries of :func:`order_maxmin` (same greedy steps, stopped early;
    O(count * n))."""
    xy = _f64(xy).reshape(-1, 2)
    perm = np.empty(int(count), dtype=np.int64)
    if _load().oracle_order_maxmin_prefix(xy.shape[0], _p(xy, _dp), int(count), _p(perm, _i64p)):
        raise ValueError("order_maxmin_prefix: count exceeds n")
    return perm


def order_morton(xy) -> np.ndarray:
    """Morton (Z-order) ordering of 16-bit cell indices over the bounding box."""
    xy = _f64(xy).reshape(-1, 2)
    perm = np.empty(xy.shape[0], dtype=np.int64)
    _load().oracle_order_morton(xy.shape[0], _p(xy, _dp), _p(perm, _i64p))
    return perm


def knn_rows(xy_ordered, m: int, rows=None) -> np.ndarray:
    """Conditioning sets (ordered indices, -1 padded) of the given ordered rows."""
    xy = _f64(xy_ordered).reshape(-1, 2)
    n = xy.shape[0]
    rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((rows.size, m), dtype=np.int32)
    rc = _load().oracle_knn_rows(n, _p(xy, _dp), m, _p(rows, _i64p), rows.size, _p(out, _i32p))
    if rc:
        raise ValueError("oracle_knn_rows: invalid arguments")
    return out


def sphere_xyz(lonlat) -> np.ndarray:
    """Unit vectors (n x 3) of (longitude, latitude) points given in degrees."""
    ll = _f64(lonlat).reshape(-1, 2)
    out = np.empty((ll.shape[0], 3), dtype=np.float64)
    _load().oracle_sphere_xyz(ll.shape[0], _p(ll, _dp), _p(out, _dp))
    return out


def gcd(a, b, radius: float) -> np.ndarray:
    """Great-circle distances (Sec. VI-C, haversine) between rows of a and b (lon, lat degrees)."""
    a = _f64(a).reshape(-1, 2)
    b = _f64(b).reshape(-1, 2)
    out = np.empty(a.shape[0], dtype=np.float64)
    _load().oracle_gcd(a.shape[0], _p(a, _dp), _p(b, _dp), float(radius), _p(out, _dp))
    return out


def knn_rows_sphere(xyz_ordered, m: int, rows=None) -> np.ndarray:
    """Conditioning sets on the sphere from ordered unit vectors, keys (chord^2, index)."""
    xyz = _f64(xyz_ordered).reshape(-1, 3)
    n = xyz.shape[0]
    rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((rows.size, m), dtype=np.int32)
    rc = _load().oracle_knn_rows_sphere(n, _p(xyz, _dp), m, _p(rows, _i64p), rows.size, _p(out, _i32p))
    if rc:
        raise ValueError("oracle_knn_rows_sphere: invalid arguments")
    return out


class OracleNotPD(RuntimeError):
    def __init__(self, row):
        super().__init__(f"conditional block not positive definite at ordered location {row}")
        self.row = row


def vecchia_rows(xy_ordered, y_ordered, m: int, theta, rows=None, nbr=None, want_grad=False,
                 return_mu_s=False, family=0, radius=None):
    """Per-location Vecchia terms (and gradients) for the given ordered rows.

    theta = (sigma2, beta, nu, tau2); family 0 = Matérn (Eq. 2), 1 = power exponential
    (Eq. 3, nu = exponent).  With ``radius`` set, the points are (longitude, latitude)
    in degrees and distances are great-circle distances on that sphere (Sec. VI-C).
    Returns an array of shape (nrows,) or (nrows, 4) = (l_i, dl_i/dsigma2, dl_i/dbeta,
    dl_i/dtau2).
    """
    xy = _f64(xy_ordered).reshape(-1, 2)
    y = _f64(y_ordered)
    n = xy.shape[0]
    rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    if nbr is None:
        nbr = knn_rows(xy, m, rows) if radius is None else knn_rows_sphere(sphere_xyz(xy), m, rows)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    th = _f64(theta)
    w = 4 if want_grad else 1
    out = np.empty((rows.size, w), dtype=np.float64)
    mu_s = np.empty((rows.size, 2), dtype=np.float64)
    bad = np.full(1, -1, dtype=np.int64)
    rc = _load().oracle_vecchia_rows(n, _p(xy, _dp), _p(y, _dp), m, _p(th, _dp), _p(rows, _i64p),
                                     rows.size, _p(nbr, _i32p), 1 if want_grad else 0, _p(out, _dp),
                                     _p(mu_s, _dp), _p(bad, _i64p), int(family),
                                     0 if radius is None else 1, 0.0 if radius is None else float(radius))
    if rc:
        raise OracleNotPD(int(bad[0]))
    res = out if want_grad else out[:, 0]
    return (res, mu_s) if return_mu_s else res


def predict(xy_obs, y_obs, xy_new, m: int, theta, family=0, radius=None):
    """Kriging from the m nearest observed locations: (mean, var, nbr) at each new point.

    var is the conditional variance of y at the new point (nugget included); nbr holds
    observed indices, nearest first, ties by index.  ``radius`` as in :func:`vecchia_rows`.
    """
    xo = _f64(xy_obs).reshape(-1, 2)
    yo = _f64(y_obs)
    xn = _f64(xy_new).reshape(-1, 2)
    th = _f64(theta)
    mean = np.empty(xn.shape[0])
    var = np.empty(xn.shape[0])
    nbr = np.empty((xn.shape[0], m), dtype=np.int32)
    rc = _load().oracle_predict(xo.shape[0], _p(xo, _dp), _p(yo, _dp), xn.shape[0], _p(xn, _dp), int(m),
                                _p(th, _dp), int(family), 0 if radius is None else 1,
                                0.0 if radius is None else float(radius), _p(mean, _dp), _p(var, _dp),
                                _p(nbr, _i32p))
    if rc == 1:
        raise ValueError("oracle_predict: invalid arguments")
    if rc:
        raise OracleNotPD(-1)
    return mean, var, nbr


def compensated_sum(v) -> np.ndarray:
    """Neumaier-compensated column sums in row order."""
    v = _f64(v)
    if v.ndim == 1:
        v = v[:, None]
    out = np.empty(v.shape[1], dtype=np.float64)
    _load().oracle_sum_columns(v.shape[0], v.shape[1], _p(v, _dp), _p(out, _dp))
    return out


def vecchia(xy_ordered, y_ordered, m: int, theta, want_grad=False, family=0, radius=None):
    """Vecchia log-likelihood over all ordered locations: l or (l, dsigma2, dbeta, dtau2)."""
    terms = vecchia_rows(xy_ordered, y_ordered, m, theta, want_grad=want_grad, family=family, radius=radius)
    s = compensated_sum(terms)
    return s if want_grad else float(s[0])


def loglik_exact(xy, y, theta, want_grad=False, family=0, radius=None):
    """Eq. (1): exact zero-mean Gaussian log-likelihood (dense, O(n^3)); ``radius`` as in
    :func:`vecchia_rows`."""
    xy = _f64(xy).reshape(-1, 2)
    y = _f64(y)
    th = _f64(theta)
    out = np.empty(1)
    g = np.empty(3)
    rc = _load().oracle_loglik_exact(xy.shape[0], _p(xy, _dp), _p(y, _dp), _p(th, _dp), _p(out, _dp),
                                     _p(g, _dp) if want_grad else None, int(family),
                                     0 if radius is None else 1, 0.0 if radius is None else float(radius))
    if rc:
        raise OracleNotPD(-1)
    return (float(out[0]), g) if want_grad else float(out[0])


def block_logdensity(S, y) -> float:
    """log N(y; 0, S) of one dense block."""
    S = _f64(S)
    y = _f64(y)
    out = np.empty(1)
    rc = _load().oracle_block_logdensity(y.size, _p(S, _dp), _p(y, _dp), _p(out, _dp))
    if rc:
        raise OracleNotPD(-1)
    return float(out[0])
