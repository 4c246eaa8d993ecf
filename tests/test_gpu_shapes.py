"""Launch shapes of small calls on the GPU.

A call over few locations widens its default lane groups (up to 16 lanes per location
while the groups would not give every SM sub-partition a warp) and spreads the groups
over every SM with fewer warps per CTA.  Neither may change what is computed: totals
and gradients match the oracle (1e-9 of the summed |l_i|, 1e-7 of the summed |dl_i|),
a repeated call returns the same bits, and every forced lane width agrees with the
default within the same tolerances.  The sizes cover the three regimes: 300 locations
(16 lanes), 2,000 (16 lanes, spread) and 6,000 (default lanes, spread at m = 30).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_07412_gb300 import datagen
from tests import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07412_gb300 import build, vecchia

    build.build()
    oracle.build()
    return vecchia


def _case(n, m):
    seed = datagen.BASE_SEED + 70 + n + m
    xy = datagen.uniform_locations(n, seed)
    theta = (1.2, 0.08, 1.5, 0.02)
    y = datagen.field_rff(xy, theta, seed + 1, features=512)
    perm = oracle.order_random(n, seed + 2)
    return xy, np.asarray(y, dtype=np.float64), theta, perm


def _close(got, want_terms):
    want = oracle.compensated_sum(want_terms)
    den = np.abs(want_terms).sum(axis=0)
    tol = np.array([W.LOGLIK_RTOL] + [W.GRAD_RTOL] * 3)
    assert np.all(np.abs(got - want) <= tol * den), (got, want)


@pytest.mark.parametrize("n", [300, 2000, 6000])
@pytest.mark.parametrize("m", [10, 30])
def test_small_calls_match_oracle_and_repeat(V, n, m, monkeypatch):
    monkeypatch.delenv("VECCHIA_LANES_PER_LOCATION", raising=False)
    xy, y, theta, perm = _case(n, m)
    p = V.Plan(xy, m, order=V.ORDER_GIVEN, perm=perm)
    yd = torch.as_tensor(y, device="cuda")
    want_terms = oracle.vecchia_rows(xy[perm], y[perm], m, theta, want_grad=True)
    a = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    b = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    assert a.tobytes() == b.tobytes()
    _close(a, want_terms)
    f = V.vecchia_loglik(p, yd, theta).cpu().numpy()
    assert abs(f[0] - oracle.compensated_sum(want_terms)[0]) <= W.LOGLIK_RTOL * np.abs(want_terms[:, 0]).sum()
    for lanes in (4, 8, 16, 32):
        if m + 1 > {4: 16, 8: 32}.get(lanes, 64):
            continue
        monkeypatch.setenv("VECCHIA_LANES_PER_LOCATION", str(lanes))
        _close(V.vecchia_loglik_grad(p, yd, theta).cpu().numpy(), want_terms)
    monkeypatch.delenv("VECCHIA_LANES_PER_LOCATION")
    p.close()
