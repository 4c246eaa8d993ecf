"""Maximum-likelihood fits driven by the adjoint kernel, checked with the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_07412_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07412_gb300 import build, vecchia

    build.build()
    oracle.build()
    return vecchia


def test_mle_recovers_parameters_and_oracle_agrees_it_is_stationary(V):
    from paper_2403_07412_gb300 import mle

    n, m = 12_000, 30
    truth = (1.0, 0.05, 1.0, 0.02)
    xy = datagen.uniform_locations(n, 61)
    y = datagen.field_rff(xy, truth, 62, features=4096)
    perm = oracle.order_random(n, 63)
    plan = V.Plan(xy, m, order=V.ORDER_GIVEN, perm=perm)
    yd = torch.as_tensor(y, device="cuda")
    res = mle.fit(plan, yd, (0.5, 0.1, 1.0, 0.1))
    assert res.converged, res.message
    s2, beta, _, t2 = res.theta
    # the draw is one realisation: loose recovery bounds
    assert 0.5 < s2 < 2.0 and 0.025 < beta < 0.1 and 0.0 <= t2 < 0.06, res.theta
    # independent check: the oracle's likelihood is no larger at the truth and its
    # gradient (sigma2, beta, tau2) is near zero at the optimum
    terms = oracle.vecchia_rows(xy[perm], y[perm], m, res.theta, want_grad=True)
    g = oracle.compensated_sum(terms)
    scale = np.abs(terms).sum(axis=0)
    for k, th in ((1, s2), (2, beta)):
        assert abs(g[k]) * th <= 1e-4 * scale[0], (k, g[k])
    if t2 > 1e-8:
        assert abs(g[3]) <= 1e-4 * scale[0] / max(t2, 1e-3)
    l_truth = oracle.vecchia(xy[perm], y[perm], m, truth)
    assert g[0] >= l_truth - 1e-9 * scale[0]


def test_mle_with_nu(V):
    from paper_2403_07412_gb300 import mle

    n, m = 8000, 20
    truth = (1.2, 0.04, 1.5, 0.01)
    xy = datagen.uniform_locations(n, 71)
    y = datagen.field_rff(xy, truth, 72, features=4096)
    plan = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=73)
    yd = torch.as_tensor(y, device="cuda")
    res = mle.fit(plan, yd, (1.0, 0.06, 1.0, 0.05), estimate_nu=True)
    assert res.converged, res.message
    assert 0.7 < res.theta[2] < 3.0, res.theta
    fixed = mle.fit(plan, yd, res.theta)  # restart at the joint optimum, nu held
    assert fixed.loglik <= res.loglik + 1e-6 * abs(res.loglik)
