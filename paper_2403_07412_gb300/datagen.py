"""Seeded synthetic inputs shaped like the paper's geospatial workloads.

This module holds only data generation: locations in the unit square and
Gaussian-field draws at them.  It computes nothing of the likelihood path, so
both the CUDA library's tests and the CPU oracle's tests may draw from it.

Workloads (the paper's numerical study uses 2-D Matérn fields with
nu in {0.5, 1.5, 2.5} at 180K/260K locations and m from 10 to 150 (Sec. VI-B,
Table II); its real data are 250K-location subsamples (Sec. VI-C), which are
not available here, so seeded synthetic fields stand in for them):

* ``uniform_locations``  — n points i.i.d. U[0,1]^2.
* ``gmm_locations``      — n points from an equal-weight Gaussian mixture in
  [0,1]^2 (means U[0.05,0.95]^2, isotropic sd log-uniform in [0.01,0.05]),
  redrawn until inside the square: a clustered layout.
* ``field_dense``        — exact zero-mean GP draw y = L z, L = chol(Sigma),
  for small n (the covariance is evaluated here with scipy's Bessel K).
* ``field_rff``          — random-Fourier-feature draw of a Matérn field plus
  nugget noise, for large n.  The spectral density of
  C(d) ∝ (d/beta)^nu K_nu(d/beta) in 2-D is ∝ (beta^-2 + |w|^2)^-(nu+1); it is
  sampled as w = z / (beta sqrt(2 g)), z ~ N(0, I_2), g ~ Gamma(nu, 1).
* ``sphere_locations``   — n (longitude, latitude) points in degrees, area-uniform
  on a latitude/longitude patch (default: a 15 x 15 degree region like the paper's
  Mississippi-basin soil data, Sec. VI-C).
* ``sphere_coords``      — 3-D coordinates (radius x unit vector) of such points, so
  that ``field_rff`` / ``field_dense`` draw fields in chordal distance on the sphere.
* ``theta_candidates``   — parameter vectors for the many-field batched mode.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2403074120


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def uniform_locations(n: int, seed: int) -> np.ndarray:
    return rng(seed).random((n, 2))


def gmm_locations(n: int, seed: int, ncomp: int = 20) -> np.ndarray:
    g = rng(seed)
    means = g.uniform(0.05, 0.95, size=(ncomp, 2))
    sds = np.exp(g.uniform(np.log(0.01), np.log(0.05), size=ncomp))
    comp = g.integers(0, ncomp, size=n)
    out = np.empty((n, 2))
    todo = np.arange(n)
    while todo.size:
        c = comp[todo]
        p = means[c] + sds[c, None] * g.standard_normal((todo.size, 2))
        ok = np.all((p >= 0.0) & (p <= 1.0), axis=1)
        out[todo[ok]] = p[ok]
        todo = todo[~ok]
    return out


def _matern_np(d: np.ndarray, sigma2: float, beta: float, nu: float) -> np.ndarray:
    from scipy.special import gamma, kv

    x = d / beta
    with np.errstate(invalid="ignore", over="ignore"):
        c = sigma2 * 2.0 ** (1.0 - nu) / gamma(nu) * x ** nu * kv(nu, x)
    c[d == 0.0] = sigma2
    c[~np.isfinite(c)] = 0.0
    return c


def field_dense(xy: np.ndarray, theta, seed: int) -> np.ndarray:
    """Exact draw of the zero-mean GP with Matérn + nugget covariance."""
    sigma2, beta, nu, tau2 = (float(t) for t in theta)
    d = np.sqrt(((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1))
    S = _matern_np(d, sigma2, beta, nu) + tau2 * np.eye(xy.shape[0])
    L = np.linalg.cholesky(S + 1e-12 * sigma2 * np.eye(xy.shape[0]))
    return L @ rng(seed).standard_normal(xy.shape[0])


def field_rff(xy: np.ndarray, theta, seed: int, features: int = 4096, device=None,
              chunk: int = 1 << 16) -> np.ndarray:
    """Random-Fourier-feature Matérn field at xy plus sqrt(tau2) white noise.

    ``device`` = a torch device string to evaluate the cosines there (fast for
    millions of points); the draws themselves always come from numpy.
    """
    sigma2, beta, nu, tau2 = (float(t) for t in theta)
    g = rng(seed)
    z = g.standard_normal((features, xy.shape[1]))
    gam = g.gamma(nu, 1.0, size=features)
    w = z / (beta * np.sqrt(2.0 * gam))[:, None]
    b = g.uniform(0.0, 2.0 * np.pi, size=features)
    eps = g.standard_normal(xy.shape[0])
    amp = np.sqrt(sigma2) * np.sqrt(2.0 / features)
    n = xy.shape[0]
    f = np.empty(n)
    if device is not None:
        import torch

        wt = torch.as_tensor(w, device=device)
        bt = torch.as_tensor(b, device=device)
        for s in range(0, n, chunk):
            p = torch.as_tensor(xy[s:s + chunk], device=device)
            f[s:s + chunk] = (torch.cos(p @ wt.T + bt).sum(1) * amp).cpu().numpy()
    else:
        for s in range(0, n, chunk // 16):
            p = xy[s:s + chunk // 16]
            f[s:s + chunk // 16] = np.cos(p @ w.T + b).sum(1) * amp
    return f + np.sqrt(tau2) * eps


def sphere_locations(n: int, seed: int, lon=(-100.0, -85.0), lat=(30.0, 45.0)) -> np.ndarray:
    """n (longitude, latitude) points in degrees, uniform in area on the patch."""
    g = rng(seed)
    lo = g.uniform(lon[0], lon[1], size=n)
    s0, s1 = np.sin(np.radians(lat[0])), np.sin(np.radians(lat[1]))
    la = np.degrees(np.arcsin(g.uniform(s0, s1, size=n)))
    return np.stack([lo, la], axis=1)


def sphere_coords(lonlat: np.ndarray, radius: float) -> np.ndarray:
    """radius x unit vectors of (longitude, latitude) points (data generation only)."""
    lam, phi = np.radians(lonlat[:, 0]), np.radians(lonlat[:, 1])
    return radius * np.stack([np.cos(phi) * np.cos(lam), np.cos(phi) * np.sin(lam), np.sin(phi)], axis=1)


def theta_candidates(nfields: int, ntheta: int, seed: int) -> np.ndarray:
    """(nfields, ntheta, 4) candidates: sigma2 ~ U[0.5,2], beta log-U[0.01,0.2],
    nu uniform on {0.5, 1.0, 1.5}, tau2 ~ U[0, 0.1]."""
    g = rng(seed)
    out = np.empty((nfields, ntheta, 4))
    out[..., 0] = g.uniform(0.5, 2.0, size=(nfields, ntheta))
    out[..., 1] = np.exp(g.uniform(np.log(0.01), np.log(0.2), size=(nfields, ntheta)))
    out[..., 2] = g.choice(np.array([0.5, 1.0, 1.5]), size=(nfields, ntheta))
    out[..., 3] = g.uniform(0.0, 0.1, size=(nfields, ntheta))
    return out


def batch_sizes(nfields: int, seed: int, n_lo: int = 10_000, n_hi: int = 500_000):
    """Field sizes log-uniform in [n_lo, n_hi] and m uniform on {10, 30, 60}."""
    g = rng(seed)
    ns = np.floor(np.exp(g.uniform(np.log(n_lo), np.log(n_hi), size=nfields))).astype(np.int64)
    ms = g.choice(np.array([10, 30, 60]), size=nfields)
    return ns, ms
