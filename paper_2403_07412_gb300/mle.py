"""Maximum-likelihood estimation of theta with the Vecchia log-likelihood and its adjoint.

The paper estimates theta by maximising the Vecchia log-likelihood with NLopt, one
likelihood evaluation per optimiser step (Sec. VI-A, VI-C).  Here every evaluation is one
call of vecchia_loglik_grad (value and d/d(sigma2, beta, tau2) from the adjoint kernel),
and the host runs L-BFGS-B (scipy) over the parameters, so the conditioning sets of the
plan are built once and reused across all iterations.  nu is either held fixed or
estimated with a central finite difference of the forward kernel.

Parameters are optimised on a log scale for sigma2, beta (and nu), which keeps them
positive, and on the natural scale for tau2 >= 0 (bounded below by zero).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import vecchia as V


@dataclass
class MLEResult:
    theta: np.ndarray          # (sigma2, beta, nu, tau2) at the optimum
    loglik: float              # Vecchia log-likelihood there
    grad: np.ndarray           # (dl/dsigma2, dl/dbeta, dl/dnu, dl/dtau2) there
    iterations: int
    evaluations: int
    converged: bool
    message: str
    history: list = field(default_factory=list)


def fit(plan: V.Plan, y: torch.Tensor, theta0, estimate_nu: bool = False, nu_step: float = 1e-6,
        max_iter: int = 200, gtol: float = 1e-7, nu_bounds=(0.05, 5.0), stream=None) -> MLEResult:
    """Maximise the Vecchia log-likelihood of field ``y`` (CUDA float64, original order)
    over theta = (sigma2, beta, nu, tau2), starting at ``theta0``."""
    from scipy.optimize import minimize

    th0 = np.asarray(theta0, dtype=np.float64)
    if th0.shape != (4,) or not np.all(np.isfinite(th0)) or th0[0] <= 0 or th0[1] <= 0 or th0[2] <= 0 or th0[3] < 0:
        raise ValueError("theta0 must be finite with sigma2, beta, nu > 0 and tau2 >= 0")
    n = plan.n
    out = torch.empty(4, dtype=torch.float64, device=y.device)
    out1 = torch.empty(1, dtype=torch.float64, device=y.device)
    history = []
    evals = [0]

    def unpack(x):
        th = th0.copy()
        th[0] = math.exp(x[0])
        th[1] = math.exp(x[1])
        th[3] = x[2]
        if estimate_nu:
            th[2] = math.exp(x[3])
        return th

    def objective(x):
        th = unpack(x)
        evals[0] += 1
        g = V.vecchia_loglik_grad(plan, y, th, out=out, stream=stream).cpu().numpy()
        if not np.all(np.isfinite(g)):
            return 1e300, np.zeros_like(x)
        # chain rule to the optimisation variables; minimise -l / n
        gx = [g[1] * th[0], g[2] * th[1], g[3]]
        if estimate_nu:
            h = nu_step * th[2]
            tp, tm = th.copy(), th.copy()
            tp[2] += h
            tm[2] -= h
            lp = V.vecchia_loglik(plan, y, tp, out=out1, stream=stream).item()
            lm = V.vecchia_loglik(plan, y, tm, out=out1, stream=stream).item()
            gx.append((lp - lm) / (2.0 * h) * th[2])
        history.append((th.copy(), float(g[0])))
        return -g[0] / n, -np.asarray(gx) / n

    x0 = [math.log(th0[0]), math.log(th0[1]), th0[3]]
    bounds = [(None, None), (None, None), (0.0, None)]
    if estimate_nu:
        x0.append(math.log(th0[2]))
        bounds.append((math.log(nu_bounds[0]), math.log(nu_bounds[1])))
    res = minimize(objective, np.asarray(x0), jac=True, method="L-BFGS-B", bounds=bounds,
                   options={"maxiter": max_iter, "gtol": gtol, "ftol": 1e-15})
    th = unpack(res.x)
    g = V.vecchia_loglik_grad(plan, y, th, out=out, stream=stream).cpu().numpy()
    h = nu_step * th[2]
    tp, tm = th.copy(), th.copy()
    tp[2] += h
    tm[2] -= h
    dnu = (V.vecchia_loglik(plan, y, tp, out=out1, stream=stream).item()
           - V.vecchia_loglik(plan, y, tm, out=out1, stream=stream).item()) / (2.0 * h)
    return MLEResult(theta=th, loglik=float(g[0]), grad=np.array([g[1], g[2], dnu, g[3]]),
                     iterations=int(res.nit), evaluations=evals[0], converged=bool(res.success),
                     message=str(res.message), history=history)
