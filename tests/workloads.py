"""Seeded workloads shaped like the paper's experiments (test and bench inputs).

Each returns (xy, y, theta, m, order) with xy in the ORIGINAL order.  Seeds derive from
datagen.BASE_SEED + the workload number.
"""
import numpy as np

from paper_2403_07412_gb300 import datagen

ORDER_RANDOM, ORDER_MAXMIN = 1, 2

# Tolerances (see the design notes): per-term and total log-likelihood within 1e-9 of
# the absolute sum of terms; gradients within 1e-7 of the absolute sum of their terms.
LOGLIK_RTOL = 1e-9
GRAD_RTOL = 1e-7


def small_exact(n=2000):
    """Plain forward: n uniform locations, exact field, nu = 0.5, tau2 = 0, m = 10."""
    seed = datagen.BASE_SEED + 1
    xy = datagen.uniform_locations(n, seed)
    theta = (1.0, 0.1, 0.5, 0.0)
    y = datagen.field_dense(xy, theta, seed + 1000)
    return xy, y, theta, 10, ORDER_RANDOM


def uniform_rff(n=100_000, device=None):
    """Plain forward: uniform, RFF field, nu = 1.5, tau2 = 0.01, m = 30."""
    seed = datagen.BASE_SEED + 2
    xy = datagen.uniform_locations(n, seed)
    theta = (1.0, 0.05, 1.5, 0.01)
    y = datagen.field_rff(xy, theta, seed + 1000, device=device)
    return xy, y, theta, 30, ORDER_RANDOM


def differentiation(n=250_000, device=None):
    """Loglik + gradient: uniform, RFF field, nu = 2.5, tau2 = 0.05, m = 60."""
    seed = datagen.BASE_SEED + 3
    xy = datagen.uniform_locations(n, seed)
    theta = (1.5, 0.03, 2.5, 0.05)
    y = datagen.field_rff(xy, theta, seed + 1000, device=device)
    return xy, y, theta, 60, ORDER_RANDOM


def scale(n=1_000_000, device=None):
    """Scale: 20-component Gaussian mixture, RFF field, general nu = 1.0, maxmin, m = 60."""
    seed = datagen.BASE_SEED + 5
    xy = datagen.gmm_locations(n, seed)
    theta = (1.0, 0.02, 1.0, 0.01)
    y = datagen.field_rff(xy, theta, seed + 1000, device=device)
    return xy, y, theta, 60, ORDER_MAXMIN


def tol_ok(got, want, rtol):
    """|sum got - sum want| <= rtol * sum |want_i| (columns treated separately)."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.abs(want).sum(axis=0)
    return np.abs(got.sum(axis=0) - want.sum(axis=0)) <= rtol * den, den
