"""GPU parity of kriging at new locations (vecchia_predict) against the CPU oracle:
conditioning sets bit for bit, conditional mean and variance within 1e-9 of
max(|value|, 1)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_07412_gb300 import datagen

pytestmark = pytest.mark.gpu
R_EARTH = 6371.0
TOL = 1e-9


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07412_gb300 import build, vecchia

    build.build()
    oracle.build()
    return vecchia


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _close(got, want):
    err = np.abs(got - want)
    bad = np.flatnonzero(err > TOL * np.maximum(np.abs(want), 1.0))
    assert bad.size == 0, (bad[:5], got[bad[:5]], want[bad[:5]])


@pytest.mark.parametrize("m,theta", [(30, (1.0, 0.05, 1.5, 0.01)), (10, (1.4, 0.1, 0.5, 0.05)),
                                     (60, (0.8, 0.03, 1.0, 0.02))])
def test_predict_matches_oracle(V, m, theta):
    n, k = 20000, 2000
    xy = datagen.uniform_locations(n, 400 + m)
    new = datagen.rng(401 + m).uniform(-0.05, 1.05, size=(k, 2))  # a few outside the observed box
    y = datagen.field_rff(xy, theta, 402 + m, features=512)
    plan = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=1)
    mean, var, nbr = V.vecchia_predict(plan, new, _dev(y), theta, return_neighbors=True)
    wm, wv, wn = oracle.predict(xy, y, new, m, theta)
    np.testing.assert_array_equal(nbr, wn)
    _close(mean.cpu().numpy(), wm)
    _close(var.cpu().numpy(), wv)


def test_predict_interpolates_observed_points(V):
    n, m = 5000, 16
    theta = (1.2, 0.05, 1.5, 0.0)
    xy = datagen.uniform_locations(n, 410)
    y = datagen.field_rff(xy, theta, 411, features=512)
    plan = V.Plan(xy, m, order=V.ORDER_MAXMIN)
    mean, var = V.vecchia_predict(plan, xy[:300], _dev(y), theta)
    _close(mean.cpu().numpy(), y[:300])
    assert np.all(np.abs(var.cpu().numpy()) <= TOL)


@pytest.mark.parametrize("family,theta", [(0, (1.0, 60.0, 0.5, 0.02)), (1, (1.1, 25.0, 0.8, 0.01))])
def test_predict_on_sphere_matches_oracle(V, family, theta):
    n, k, m = 5000, 500, 20
    ll = datagen.sphere_locations(n + k, 420)
    y = datagen.field_rff(datagen.sphere_coords(ll[:n], R_EARTH), (1.0, 60.0, 0.5, 0.02), 421, features=512)
    plan = V.Plan(ll[:n], m, order=V.ORDER_RANDOM, seed=2, radius=R_EARTH)
    if family == 1:
        plan.set_kernel(V.KERNEL_POWEXP)
    mean, var, nbr = V.vecchia_predict(plan, ll[n:], _dev(y), theta, return_neighbors=True)
    wm, wv, wn = oracle.predict(ll[:n], y, ll[n:], m, theta, family=family, radius=R_EARTH)
    np.testing.assert_array_equal(nbr, wn)
    _close(mean.cpu().numpy(), wm)
    _close(var.cpu().numpy(), wv)


def test_predict_rejections(V):
    xy = datagen.uniform_locations(500, 430)
    y = _dev(np.zeros(500))
    with pytest.raises(V.VecchiaError):
        V.vecchia_predict(V.Plan(xy, 80), xy[:5], y, (1.0, 0.1, 0.5, 0.0))  # m beyond the warp kernels
    with pytest.raises(V.VecchiaError):
        V.vecchia_predict(V.Plan(xy, 10), np.array([[0.5, np.nan]]), y, (1.0, 0.1, 0.5, 0.0))
    ll = datagen.sphere_locations(500, 431)
    with pytest.raises(V.VecchiaError):
        V.vecchia_predict(V.Plan(ll, 10, radius=R_EARTH), np.array([[0.0, 95.0]]), y, (1.0, 50.0, 0.5, 0.0))
