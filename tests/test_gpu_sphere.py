"""GPU parity on the sphere (Sec. VI-C great-circle distances): the CUDA library's
sphere plans against the CPU oracle's haversine path.

Neighbour sets must match bit for bit (keys: squared chord of the unit vectors);
log-likelihood terms within 1e-9 and gradient terms within 1e-7, as for the plane.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_07412_gb300 import datagen
from tests import workloads as W

pytestmark = pytest.mark.gpu
R_EARTH = 6371.0


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


def _check_terms(got, want):
    got, want = np.asarray(got), np.asarray(want)
    err = np.abs(got[:, 0] - want[:, 0])
    bad = np.flatnonzero(err > W.LOGLIK_RTOL * np.maximum(np.abs(want[:, 0]), 1.0))
    assert bad.size == 0, (bad[:5], got[bad[:5], 0], want[bad[:5], 0])
    scale = np.abs(want[:, 1:]).mean(axis=0)
    err = np.abs(got[:, 1:] - want[:, 1:])
    bad = np.argwhere(err > W.GRAD_RTOL * np.maximum(np.abs(want[:, 1:]), scale))
    assert bad.size == 0, (bad[:5], got[bad[:5, 0]], want[bad[:5, 0]])


def _field(ll, theta, seed):
    xyz = datagen.sphere_coords(ll, R_EARTH)
    return datagen.field_rff(xyz, theta, seed, features=512)


@pytest.mark.parametrize("region,n,m", [("patch", 20000, 30), ("globe", 6000, 12), ("patch", 3000, 100)])
def test_sphere_neighbours_bit_exact(V, region, n, m):
    ll = (datagen.sphere_locations(n, 200 + m) if region == "patch"
          else datagen.sphere_locations(n, 201, lon=(-180.0, 180.0), lat=(-90.0, 90.0)))
    p = V.Plan(ll, m, order=V.ORDER_RANDOM, seed=7, radius=R_EARTH)
    perm = p.perm()
    np.testing.assert_array_equal(perm, oracle.order_random(n, 7))
    xyz = oracle.sphere_xyz(ll[perm])
    np.testing.assert_array_equal(p.neighbors(), oracle.knn_rows_sphere(xyz, m))


@pytest.mark.parametrize("family,theta,region", [
    (0, (1.0, 60.0, 0.5, 0.02), "patch"),
    (0, (1.4, 40.0, 1.5, 0.05), "patch"),
    (1, (1.1, 25.0, 0.8, 0.01), "patch"),
    (0, (1.0, 900.0, 0.5, 0.05), "globe"),   # long chords: the FP64 asin branch
])
def test_sphere_terms_match_oracle(V, family, theta, region):
    n, m = 3000, 20
    ll = (datagen.sphere_locations(n, 210) if region == "patch"
          else datagen.sphere_locations(n, 211, lon=(-180.0, 180.0), lat=(-90.0, 90.0)))
    y = _field(ll, (1.0, theta[1] if family == 0 else 30.0, 0.5, 0.02), 212)
    perm = oracle.order_random(n, 213)
    p = V.Plan(ll, m, order=V.ORDER_GIVEN, perm=perm, radius=R_EARTH)
    if family == 1:
        p.set_kernel(V.KERNEL_POWEXP)
    yd = _dev(y)
    want = oracle.vecchia_rows(ll[perm], y[perm], m, theta, want_grad=True, family=family, radius=R_EARTH)
    _check_terms(V.vecchia_loglik_terms(p, yd, theta, want_grad=True).cpu().numpy(), want)
    tot = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    ref = oracle.compensated_sum(want)
    assert abs(tot[0] - ref[0]) <= W.LOGLIK_RTOL * np.abs(want[:, 0]).sum()
    for k in (1, 2, 3):
        assert abs(tot[k] - ref[k]) <= W.GRAD_RTOL * np.abs(want[:, k]).sum(), (k, tot[k], ref[k])
    fwd = V.vecchia_loglik(p, yd, theta).item()
    assert abs(fwd - ref[0]) <= W.LOGLIK_RTOL * np.abs(want[:, 0]).sum()


def test_sphere_full_conditioning_equals_exact(V):
    # m = n - 1 on the sphere: the Vecchia product is the dense Eq. (1) likelihood.
    n = 120
    theta = (1.2, 80.0, 0.5, 0.03)
    ll = datagen.sphere_locations(n, 220)
    y = _field(ll, theta, 221)
    p = V.Plan(ll, n - 1, order=V.ORDER_RANDOM, seed=3, radius=R_EARTH)
    got = V.vecchia_loglik_grad(p, _dev(y), theta).cpu().numpy()
    ex, gex = oracle.loglik_exact(ll, y, theta, want_grad=True, radius=R_EARTH)
    assert abs(got[0] - ex) <= 1e-9 * abs(ex)
    np.testing.assert_allclose(got[1:], gex, rtol=1e-7, atol=1e-7 * np.abs(gex).max())


def test_sphere_large_m_matches_oracle(V):
    n, m = 1500, 80
    theta = (1.0, 50.0, 0.5, 0.02)
    ll = datagen.sphere_locations(n, 230)
    y = _field(ll, theta, 231)
    perm = oracle.order_random(n, 232)
    p = V.Plan(ll, m, order=V.ORDER_GIVEN, perm=perm, radius=R_EARTH)
    want = oracle.vecchia_rows(ll[perm], y[perm], m, theta, want_grad=True, radius=R_EARTH)
    _check_terms(V.vecchia_loglik_terms(p, _dev(y), theta, want_grad=True).cpu().numpy(), want)


def test_sphere_plan_rejections(V):
    ll = datagen.sphere_locations(200, 240)
    for order in (V.ORDER_MAXMIN, V.ORDER_MORTON):
        with pytest.raises(V.VecchiaError):
            V.Plan(ll, 10, order=order, radius=R_EARTH)
    bad = ll.copy()
    bad[3, 1] = 91.0
    with pytest.raises(V.VecchiaError):
        V.Plan(bad, 10, radius=R_EARTH)
    with pytest.raises(V.VecchiaError):
        V.Plan(ll, 10, radius=-1.0)
    p = V.Plan(ll, 10, radius=R_EARTH)
    V.vecchia_batched_prepare([0.5])
    b = V.Batch([p], [_dev(np.zeros(200))], 1, want_grad=False)
    with pytest.raises(V.VecchiaError):
        b.run(_dev(np.array([[[1.0, 50.0, 0.5, 0.0]]])))


def test_sphere_gradient_central_differences(V):
    # dl/d(sigma2, beta, tau2) through the asin series against central differences of
    # the GPU forward (h = 1e-6 relative, as for the planar path).
    n, m = 4000, 25
    theta = np.array([1.1, 45.0, 0.5, 0.03])
    ll = datagen.sphere_locations(n, 250)
    y = _field(ll, tuple(theta), 251)
    p = V.Plan(ll, m, order=V.ORDER_RANDOM, seed=4, radius=R_EARTH)
    yd = _dev(y)
    g = V.vecchia_loglik_grad(p, yd, tuple(theta)).cpu().numpy()
    for k, idx in ((1, 0), (2, 1), (3, 3)):
        h = 1e-6 * theta[idx]
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += h
        tm[idx] -= h
        fd = (V.vecchia_loglik(p, yd, tuple(tp)).item() - V.vecchia_loglik(p, yd, tuple(tm)).item()) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(g[0]), (k, g[k], fd)

