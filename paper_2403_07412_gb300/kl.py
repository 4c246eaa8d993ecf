"""Kullback-Leibler divergence of the Vecchia approximation from the exact Gaussian (Eq. 5).

For zero-mean Gaussians N_0 = N(0, Sigma) and its Vecchia approximation N_a, Eq. (5)
gives D_KL(N_0 || N_a) = l_0(theta; 0) - l_a(theta; 0): the exact and the approximated
log-likelihoods at y = 0 (Sec. IV-B).  l_a comes from the Vecchia kernel with a zero
field; l_0 = -n/2 log(2 pi) - 1/2 log|Sigma| needs the dense covariance, whose entries are
evaluated by the library's own covariance code (vecchia_matern) and whose log-determinant
is taken from a dense FP64 Cholesky on the GPU, so this is a small-n study tool
(n up to a few tens of thousands), as in the paper's numerical study (Sec. VI-B).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import vecchia as V


def exact_loglik_zero(xy, theta, device="cuda", block=4096) -> float:
    """l_0(theta; 0) for locations xy (n x 2) with the Matérn + nugget covariance."""
    xy_t = torch.as_tensor(np.ascontiguousarray(xy, dtype=np.float64), device=device)
    n = xy_t.shape[0]
    S = torch.empty((n, n), dtype=torch.float64, device=device)
    for r in range(0, n, block):
        d = torch.cdist(xy_t[r:r + block], xy_t).contiguous()
        S[r:r + block] = V.vecchia_matern(d.reshape(-1), theta, with_dbeta=False).reshape(d.shape)
    S.diagonal().add_(float(theta[3]))
    L = torch.linalg.cholesky(S)
    logdet = 2.0 * torch.log(torch.diagonal(L)).sum().item()
    return -0.5 * n * math.log(2.0 * math.pi) - 0.5 * logdet


def vecchia_loglik_zero(plan: V.Plan, theta, device="cuda") -> float:
    """l_a(theta; 0): the Vecchia log-likelihood of a zero field."""
    y0 = torch.zeros(plan.n, dtype=torch.float64, device=device)
    return V.vecchia_loglik(plan, y0, theta).item()


def kl_curve(xy, theta, ms, order=V.ORDER_RANDOM, seed=0, device="cuda"):
    """[(m, D_KL)] for the conditioning sizes ms under one ordering (Eq. 5)."""
    l0 = exact_loglik_zero(xy, theta, device=device)
    out = []
    for m in ms:
        plan = V.Plan(xy, int(m), order=order, seed=seed)
        out.append((int(m), l0 - vecchia_loglik_zero(plan, theta, device=device)))
        plan.close()
    return out
