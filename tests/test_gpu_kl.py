"""Eq. (5) KL study at small n: exact l_0 against the oracle, KL >= 0 and shrinking in m,
for random and Morton orderings."""
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


def test_exact_zero_field_loglik_matches_oracle(V):
    from paper_2403_07412_gb300 import kl

    xy = datagen.uniform_locations(600, 81)
    theta = (1.0, 0.1, 1.5, 0.01)
    l0 = kl.exact_loglik_zero(xy, theta)
    want = oracle.loglik_exact(xy, np.zeros(600), theta)
    assert abs(l0 - want) <= 1e-9 * abs(want)


@pytest.mark.parametrize("nu,beta", [(0.5, 0.078809), (1.5, 0.052537), (2.5, 0.042869)])
def test_kl_nonnegative_and_decreasing(V, nu, beta):
    # Table II ranges (effective range 0.3) at n = 3000, random and Morton orderings.
    from paper_2403_07412_gb300 import kl

    xy = datagen.uniform_locations(3000, 82)
    theta = (1.0, beta, nu, 1e-4)  # a small nugget keeps the smooth dense covariance factorable
    ms = [5, 10, 20, 40, 63]
    for order in (V.ORDER_RANDOM, V.ORDER_MORTON):
        curve = kl.kl_curve(xy, theta, ms, order=order, seed=3)
        vals = np.array([v for _, v in curve])
        scale = 1e-8 * 3000
        assert np.all(vals >= -scale), (order, vals)
        assert np.all(np.diff(vals) <= scale), (order, vals)
    # the Vecchia part at y = 0 agrees with the oracle under the same (oracle) ordering
    perm = oracle.order_random(3000, 5)
    p = V.Plan(xy, 20, order=V.ORDER_GIVEN, perm=perm)
    la = kl.vecchia_loglik_zero(p, theta)
    want = oracle.vecchia(xy[perm], np.zeros(3000), 20, theta)
    assert abs(la - want) <= 1e-9 * 3000 * 2
