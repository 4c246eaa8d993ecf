"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Neighbour sets and orderings must match bit for bit.  Log-likelihood terms must agree
within 1e-9 (relative to max(|l_i|, 1) per term, and to sum |l_i| for totals), gradient
terms within 1e-7 (relative to the column's sum of |terms| for totals).  Full-size
workloads are checked on sampled rows, which the oracle recomputes from scratch
(its own ordering, its own neighbour search).
"""
import math

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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _plan_given(V, xy, m, perm):
    return V.Plan(xy, m, order=V.ORDER_GIVEN, perm=perm)


def _check_terms(got, want, grad=False):
    got = np.asarray(got)
    want = np.asarray(want)
    if not grad:
        err = np.abs(got - want)
        bound = W.LOGLIK_RTOL * np.maximum(np.abs(want), 1.0)
        bad = np.flatnonzero(err > bound)
        assert bad.size == 0, (bad[:5], got[bad[:5]], want[bad[:5]])
        return
    _check_terms(got[:, 0], want[:, 0])
    scale = np.abs(want[:, 1:]).mean(axis=0)
    err = np.abs(got[:, 1:] - want[:, 1:])
    bound = W.GRAD_RTOL * np.maximum(np.abs(want[:, 1:]), scale)
    bad = np.argwhere(err > bound)
    assert bad.size == 0, (bad[:5], got[bad[:5, 0]], want[bad[:5, 0]])


# ------------------------------------------------------------------ covariance
@pytest.mark.parametrize("nu", [0.5, 1.0, 1.5, 2.5, 0.3, 0.8, 3.7])
def test_matern_matches_oracle(V, nu):
    rng = np.random.default_rng(3)
    beta, sigma2 = 0.05, 1.3
    d = np.concatenate([[0.0, 1e-12, 1e-9, 2e-7, 1e-6], beta * np.exp(rng.uniform(-14, 6.5, 20000)),
                        [beta * 2.0 ** 9.9, beta * 1024.0, beta * 5000.0]])
    c, dc = V.vecchia_matern(_dev(d), (sigma2, beta, nu, 0.0))
    c, dc = c.cpu().numpy(), dc.cpu().numpy()
    # the d -> 0 limit of Eq. (2) is sigma2 (the oracle's Bessel product is inexact there)
    c0 = V.vecchia_matern(_dev(np.array([1e-300, 1e-200])), (sigma2, beta, nu, 0.0), with_dbeta=False)
    assert c0.cpu().numpy().tolist() == [sigma2, sigma2]
    want = oracle.matern(d, sigma2, beta, nu)
    wantd = oracle.matern_dbeta(d, sigma2, beta, nu)
    # Both sides are a few ulp from the true value: the oracle multiplies five rounded
    # factors (pow, tgamma, K_nu, ...), the table adds its fit (< 1e-16) and Horner rounding.
    err = np.abs(c - want)
    assert np.all(err <= 4e-15 * sigma2), (err.max(), d[np.argmax(err)])
    # dC/dbeta is a double-float evaluation whose high-order tail (c5..c8) is plain FP32:
    # ~1e-14 relative where the correlation is not small, up to ~1e-8 relative where
    # |dC/dbeta| is tiny against its largest value.  What the gradient needs is an
    # absolute error small against the largest |dC/dbeta|, so the bound is 2e-9
    # relative plus 1e-10 of the largest magnitude.
    ratio = np.abs(dc - wantd) / (2e-9 * np.abs(wantd) + 1e-10 * np.abs(wantd).max())
    k = int(np.argmax(ratio))
    assert ratio[k] <= 1.0, (ratio[k], d[k] / beta, dc[k], wantd[k])


# ------------------------------------------------------------------ orderings and kNN
def test_random_ordering_bit_exact(V):
    xy = datagen.uniform_locations(50_000, 1)
    p = V.Plan(xy, 5, order=V.ORDER_RANDOM, seed=12345)
    np.testing.assert_array_equal(p.perm(), oracle.order_random(50_000, 12345))


@pytest.mark.parametrize("kind,n", [("uniform", 3000), ("gmm", 20_000), ("grid", 900)])
def test_maxmin_ordering_bit_exact(V, kind, n):
    if kind == "uniform":
        xy = datagen.uniform_locations(n, 2)
    elif kind == "gmm":
        xy = datagen.gmm_locations(n, 3)
    else:
        g = np.linspace(0.0, 1.0, 30)
        xy = np.array([[a, b] for b in g for a in g])
    p = V.Plan(xy, 4, order=V.ORDER_MAXMIN)
    np.testing.assert_array_equal(p.perm(), oracle.order_maxmin(xy))


@pytest.mark.parametrize("kind", ["uniform", "gmm"])
def test_morton_ordering_bit_exact(V, kind):
    xy = datagen.uniform_locations(30_000, 7) if kind == "uniform" else datagen.gmm_locations(30_000, 8)
    p = V.Plan(xy, 10, order=V.ORDER_MORTON)
    np.testing.assert_array_equal(p.perm(), oracle.order_morton(xy))


@pytest.mark.parametrize("n,m,kind", [(2000, 10, "uniform"), (5000, 63, "gmm"), (7, 10, "uniform"),
                                      (1, 3, "uniform"), (3000, 30, "dups"), (40_000, 60, "gmm")])
def test_knn_bit_exact(V, n, m, kind):
    if kind == "uniform":
        xy = datagen.uniform_locations(n, 4)
    elif kind == "gmm":
        xy = datagen.gmm_locations(n, 5)
    else:
        xy = datagen.uniform_locations(n, 6)
        xy[1::7] = xy[0::7][: xy[1::7].shape[0]]          # exact duplicates
        xy[2::11, 0] = 0.5                                # collinear points
    perm = oracle.order_random(n, 77)
    p = _plan_given(V, xy, m, perm)
    np.testing.assert_array_equal(p.perm(), perm)
    np.testing.assert_array_equal(p.neighbors(), oracle.knn_rows(xy[perm], m))


def test_knn_full_size_sampled(V):
    xy, y, theta, m, order = W.uniform_rff(100_000)
    perm = oracle.order_random(xy.shape[0], 9)
    p = _plan_given(V, xy, m, perm)
    rows = np.sort(np.random.default_rng(0).choice(xy.shape[0], 3000, replace=False))
    rows[:3] = [0, 1, m]
    np.testing.assert_array_equal(p.neighbors()[rows], oracle.knn_rows(xy[perm], m, rows))


# ------------------------------------------------------------------ log-likelihood
def test_small_exact_workload_full_parity(V):
    xy, y, theta, m, order = W.small_exact()
    n = xy.shape[0]
    perm = oracle.order_random(n, datagen.BASE_SEED + 1)
    p = _plan_given(V, xy, m, perm)
    yd = _dev(y)
    terms = V.vecchia_loglik_terms(p, yd, theta).cpu().numpy()
    want = oracle.vecchia_rows(xy[perm], y[perm], m, theta)
    _check_terms(terms, want)
    tot = float(V.vecchia_loglik(p, yd, theta).cpu()[0])
    assert abs(tot - oracle.compensated_sum(want)[0]) <= W.LOGLIK_RTOL * np.abs(want).sum()


def test_uniform_rff_full_parity(V):
    xy, y, theta, m, order = W.uniform_rff()
    n = xy.shape[0]
    perm = oracle.order_random(n, datagen.BASE_SEED + 2)
    p = _plan_given(V, xy, m, perm)
    yd = _dev(y)
    terms = V.vecchia_loglik_terms(p, yd, theta).cpu().numpy()
    want = oracle.vecchia_rows(xy[perm], y[perm], m, theta)
    _check_terms(terms, want)
    tot = float(V.vecchia_loglik(p, yd, theta).cpu()[0])
    assert abs(tot - oracle.compensated_sum(want)[0]) <= W.LOGLIK_RTOL * np.abs(want).sum()


@pytest.mark.parametrize("theta", [(1.5, 0.03, 2.5, 0.05), (1.0, 0.1, 0.5, 0.0), (0.7, 0.05, 1.0, 0.02),
                                   (2.0, 0.2, 0.3, 0.1)])
def test_gradient_terms_parity(V, theta):
    n, m = 4000, 20
    xy = datagen.uniform_locations(n, 8)
    y = datagen.field_rff(xy, theta, 9, features=1024)
    perm = oracle.order_random(n, 10)
    p = _plan_given(V, xy, m, perm)
    yd = _dev(y)
    got = V.vecchia_loglik_terms(p, yd, theta, want_grad=True).cpu().numpy()
    want = oracle.vecchia_rows(xy[perm], y[perm], m, theta, want_grad=True)
    _check_terms(got, want, grad=True)
    tot = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    ok, den = W.tol_ok(tot[None, :], oracle.compensated_sum(want)[None, :], 0.0)
    ref = oracle.compensated_sum(want)
    assert abs(tot[0] - ref[0]) <= W.LOGLIK_RTOL * np.abs(want[:, 0]).sum()
    for k in (1, 2, 3):
        assert abs(tot[k] - ref[k]) <= W.GRAD_RTOL * np.abs(want[:, k]).sum(), (k, tot[k], ref[k])


def test_gradient_central_differences(V):
    # The kernel's adjoint against central finite differences of its own forward (h = 1e-6 rel).
    xy, y, theta, m, order = W.differentiation(60_000)
    p = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=3)
    yd = _dev(y)
    g = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    for k, ti in ((1, 0), (2, 1), (3, 3)):
        h = 1e-6 * theta[ti]
        tp, tm = list(theta), list(theta)
        tp[ti] += h
        tm[ti] -= h
        fd = (float(V.vecchia_loglik(p, yd, tp).cpu()[0]) - float(V.vecchia_loglik(p, yd, tm).cpu()[0])) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(g[0]), (k, g[k], fd)


@pytest.mark.parametrize("maker,rows_n,grad", [(W.differentiation, 1500, True), (W.scale, 1000, True)])
def test_full_size_sampled_terms(V, maker, rows_n, grad):
    xy, y, theta, m, order = maker(device="cuda")
    n = xy.shape[0]
    perm = oracle.order_random(n, 4242)
    p = _plan_given(V, xy, m, perm)
    yd = _dev(y)
    terms = V.vecchia_loglik_terms(p, yd, theta, want_grad=grad).cpu().numpy()
    rows = np.sort(np.random.default_rng(1).choice(n, rows_n, replace=False))
    rows[:4] = [0, 1, 2, m + 1]
    want = oracle.vecchia_rows(xy[perm], y[perm], m, theta, rows=rows, want_grad=grad)
    _check_terms(terms[rows], want, grad=grad)
    # totals are the sums of the terms (same kernel, summed on the device)
    tot = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    assert abs(tot[0] - terms[:, 0].sum()) <= W.LOGLIK_RTOL * np.abs(terms[:, 0]).sum()


def test_scale_workload_maxmin_properties(V):
    # Full-size clustered layout with maxmin ordering: sampled maxmin property checked
    # from scratch, and total = sum of terms.
    xy, y, theta, m, order = W.scale(device="cuda")
    n = xy.shape[0]
    p = V.Plan(xy, m, order=V.ORDER_MAXMIN)
    perm = p.perm()
    assert np.array_equal(np.sort(perm), np.arange(n))
    pts = xy[perm]
    rng = np.random.default_rng(5)
    # d_k = squared distance of the k-th point to the points before it; maxmin picks the
    # largest such value among all points not yet chosen.
    ks = np.sort(rng.choice(np.arange(1, n), 60, replace=False))
    for k in ks[:20]:
        prev = pts[:k]
        dk = ((prev - pts[k]) ** 2).sum(1).min()
        later = pts[k + 1 + rng.choice(n - k - 1, min(200, n - k - 1), replace=False)]
        dl = np.array([((prev - q) ** 2).sum(1).min() for q in later])
        assert np.all(dl <= dk), k
    yd = _dev(y)
    terms = V.vecchia_loglik_terms(p, yd, theta).cpu().numpy()
    tot = float(V.vecchia_loglik(p, yd, theta).cpu()[0])
    assert np.all(np.isfinite(terms))
    assert abs(tot - terms.sum()) <= W.LOGLIK_RTOL * np.abs(terms).sum()


# ------------------------------------------------------------------ edge cases
def test_single_location_and_m_beyond_n(V):
    theta = (1.3, 0.1, 1.0, 0.2)
    xy = np.array([[0.3, 0.4]])
    y = np.array([0.7])
    p = V.Plan(xy, 5)
    got = float(V.vecchia_loglik(p, _dev(y), theta).cpu()[0])
    want = -0.5 * 0.49 / 1.5 - 0.5 * math.log(1.5) - 0.5 * math.log(2 * math.pi)
    assert abs(got - want) < 1e-14
    xy = datagen.uniform_locations(6, 1)
    y = np.linspace(-1, 1, 6)
    p = V.Plan(xy, 40)
    perm = p.perm()
    got = V.vecchia_loglik_terms(p, _dev(y), theta).cpu().numpy()
    want = oracle.vecchia_rows(xy[perm], y[perm], 40, theta)
    _check_terms(got, want)
    # m >= n - 1 reproduces the exact likelihood, Eq. (1)
    assert abs(got.sum() - oracle.loglik_exact(xy, y, theta)) < 1e-12


def test_max_m_and_near_coincident_points(V):
    n, m = 3000, 63
    xy = datagen.gmm_locations(n, 11)
    xy[5::50] = xy[4::50] + 1e-9      # u far below the table range
    xy[7::50] = xy[6::50]              # exact duplicates (nugget keeps blocks PD)
    theta = (1.0, 0.05, 1.0, 0.05)
    y = datagen.field_rff(xy, theta, 12, features=512)
    perm = oracle.order_random(n, 13)
    p = _plan_given(V, xy, m, perm)
    got = V.vecchia_loglik_terms(p, _dev(y), theta, want_grad=True).cpu().numpy()
    want = oracle.vecchia_rows(xy[perm], y[perm], m, theta, want_grad=True)
    _check_terms(got, want, grad=True)
    for nu in (0.5, 1.5, 2.0):
        th = (1.0, 0.05, nu, 0.05)
        got = V.vecchia_loglik_terms(p, _dev(y), th).cpu().numpy()
        _check_terms(got, oracle.vecchia_rows(xy[perm], y[perm], m, th))


def test_not_positive_definite_reports_location(V):
    xy = datagen.uniform_locations(200, 14)
    perm = oracle.order_random(200, 15)
    xy[perm[57]] = xy[perm[3]]          # duplicate of an earlier point, no nugget
    p = _plan_given(V, xy, 8, perm)
    y = _dev(np.linspace(-1, 1, 200))
    out = V.vecchia_loglik(p, y, (1.0, 0.1, 0.5, 0.0)).cpu().numpy()
    assert np.isnan(out[0])
    assert p.last_error_location() == 57
    ok = V.vecchia_loglik(p, y, (1.0, 0.1, 0.5, 0.01)).cpu().numpy()
    assert np.isfinite(ok[0]) and p.last_error_location() == -1


def test_invalid_theta_rejected(V):
    xy = datagen.uniform_locations(50, 1)
    p = V.Plan(xy, 5)
    y = _dev(np.zeros(50))
    for th in [(0.0, 0.1, 0.5, 0.0), (1.0, -1.0, 0.5, 0.0), (1.0, 0.1, 0.0, 0.0), (1.0, 0.1, 0.5, -1e-3),
               (float("nan"), 0.1, 0.5, 0.0), (1.0, float("inf"), 0.5, 0.0)]:
        with pytest.raises(V.VecchiaError) as e:
            V.vecchia_loglik(p, y, th)
        assert e.value.code == V.EINVAL


def test_autograd_function(V):
    xy = datagen.uniform_locations(3000, 21)
    theta0 = (1.2, 0.07, 1.5, 0.03)
    y = datagen.field_rff(xy, theta0, 22, features=512)
    p = V.Plan(xy, 15)
    th = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    ll = V.VecchiaLogLik.apply(th, p, _dev(y))
    ll.backward()
    g = V.vecchia_loglik_grad(p, _dev(y), theta0).cpu().numpy()
    assert abs(float(ll) - g[0]) == 0.0
    np.testing.assert_allclose(th.grad.numpy()[[0, 1, 3]], g[1:], rtol=0, atol=0)
    perm = p.perm()
    h = 1e-6 * theta0[2]
    lp = oracle.vecchia(xy[perm], y[perm], 15, (1.2, 0.07, 1.5 + h, 0.03))
    lm = oracle.vecchia(xy[perm], y[perm], 15, (1.2, 0.07, 1.5 - h, 0.03))
    assert abs(th.grad.numpy()[2] - (lp - lm) / (2 * h)) <= 1e-5 * abs((lp - lm) / (2 * h)) + 1e-6


@pytest.mark.parametrize("lanes", [4, 8, 16, 32])
@pytest.mark.parametrize("m", [10, 15, 31, 63])
def test_lanes_per_location_shapes_match_oracle(V, lanes, m, monkeypatch):
    # Every launch shape (32/lanes locations per warp) gives the oracle's terms, including
    # the ragged last round of locations and the short early conditioning sets.  Four lanes
    # serve blocks of at most 16 rows and eight at most 32; beyond that the launch widens
    # the group (m = 15 and 31 are those edges).
    monkeypatch.setenv("VECCHIA_LANES_PER_LOCATION", str(lanes))
    n = 1531
    theta = (1.1, 0.06, 1.5, 0.03)
    xy = datagen.gmm_locations(n, 40 + m)
    y = datagen.field_rff(xy, theta, 41 + m, features=512)
    perm = oracle.order_random(n, 42 + m)
    p = _plan_given(V, xy, m, perm)
    yd = _dev(y)
    want = oracle.vecchia_rows(xy[perm], y[perm], m, theta, want_grad=True)
    _check_terms(V.vecchia_loglik_terms(p, yd, theta, want_grad=True).cpu().numpy(), want, grad=True)
    _check_terms(V.vecchia_loglik_terms(p, yd, theta).cpu().numpy(), want[:, 0])
    tot = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    ref = oracle.compensated_sum(want)
    assert abs(tot[0] - ref[0]) <= W.LOGLIK_RTOL * np.abs(want[:, 0]).sum()
    for k in (1, 2, 3):
        assert abs(tot[k] - ref[k]) <= W.GRAD_RTOL * np.abs(want[:, k]).sum()


def test_autotune_records_a_shape(V):
    xy = datagen.uniform_locations(20_000, 50)
    theta = (1.0, 0.05, 1.0, 0.02)
    y = datagen.field_rff(xy, theta, 51, features=512)
    p = V.Plan(xy, 30)
    yd = _dev(y)
    before = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    g, w = V.vecchia_autotune(p, yd, theta, want_grad=True)
    assert g in (8, 16, 32) and 1 <= w <= 13  # 31 rows: too many for 4 lanes
    after = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    terms = V.vecchia_loglik_terms(p, yd, theta, want_grad=True).cpu().numpy()
    den = np.abs(terms).sum(axis=0)
    assert abs(after[0] - before[0]) <= W.LOGLIK_RTOL * den[0]
    for k in (1, 2, 3):
        assert abs(after[k] - before[k]) <= W.GRAD_RTOL * den[k]
    # m beyond the warp kernels: nothing to time, the CTA size chosen by occupancy
    q = V.Plan(xy[:3000], 100)
    t, wq = V.vecchia_autotune(q, _dev(y[:3000]), theta, want_grad=False)
    assert t in (128, 256) and wq == t // 32


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5, 2.0])
def test_powexp_covariance_matches_oracle(V, alpha):
    rng = np.random.default_rng(5)
    beta, sigma2 = 0.07, 1.1
    d = np.concatenate([[0.0, 1e-12, 1e-7], np.exp(rng.uniform(-16, 2.5, 20000))])
    c, dc = V.vecchia_covariance(V.KERNEL_POWEXP, _dev(d), (sigma2, beta, alpha, 0.0))
    c, dc = c.cpu().numpy(), dc.cpu().numpy()
    want = oracle.powexp(d, sigma2, beta, alpha)
    wantd = oracle.powexp_dbeta(d, sigma2, beta, alpha)
    err = np.abs(c - want)
    assert np.all(err <= 4e-15 * sigma2), (err.max(), d[np.argmax(err)])
    ratio = np.abs(dc - wantd) / (2e-9 * np.abs(wantd) + 1e-10 * np.abs(wantd).max())
    k = int(np.argmax(ratio))
    assert ratio[k] <= 1.0, (ratio[k], d[k], dc[k], wantd[k])
    with pytest.raises(V.VecchiaError):
        V.vecchia_covariance(V.KERNEL_POWEXP, _dev(d[:5]), (sigma2, beta, 2.5, 0.0))


@pytest.mark.parametrize("alpha", [0.7, 1.0, 1.9])
def test_powexp_likelihood_terms_match_oracle(V, alpha):
    n, m = 3000, 25
    theta = (1.2, 0.03 ** alpha, alpha, 0.02)
    xy = datagen.gmm_locations(n, 92)
    y = datagen.field_rff(xy, (1.0, 0.03, 0.5, 0.02), 93, features=512)
    perm = oracle.order_random(n, 94)
    p = _plan_given(V, xy, m, perm)
    p.set_kernel(V.KERNEL_POWEXP)
    yd = _dev(y)
    want = oracle.vecchia_rows(xy[perm], y[perm], m, theta, want_grad=True, family=1)
    _check_terms(V.vecchia_loglik_terms(p, yd, theta, want_grad=True).cpu().numpy(), want, grad=True)
    tot = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    ref = oracle.compensated_sum(want)
    assert abs(tot[0] - ref[0]) <= W.LOGLIK_RTOL * np.abs(want[:, 0]).sum()
    for k in (1, 2, 3):
        assert abs(tot[k] - ref[k]) <= W.GRAD_RTOL * np.abs(want[:, k]).sum(), (k, tot[k], ref[k])


@pytest.mark.parametrize("m", [64, 67, 90, 150])
def test_large_conditioning_sets_match_oracle(V, m):
    # m beyond the warp kernels: one CTA per location (the paper runs m up to 150).  The
    # m neighbour columns are eliminated four at a time, then two, then one: m = 64, 90
    # and 150 leave no column, two and two; m = 67 leaves three (a pair and a single).
    n = 1200
    theta = (1.3, 0.08, 1.0, 0.02)
    xy = datagen.uniform_locations(n, 100 + m)
    y = datagen.field_rff(xy, theta, 101 + m, features=512)
    perm = oracle.order_random(n, 102 + m)
    p = _plan_given(V, xy, m, perm)
    np.testing.assert_array_equal(p.neighbors(), oracle.knn_rows(xy[perm], m))
    yd = _dev(y)
    want = oracle.vecchia_rows(xy[perm], y[perm], m, theta, want_grad=True)
    _check_terms(V.vecchia_loglik_terms(p, yd, theta, want_grad=True).cpu().numpy(), want, grad=True)
    _check_terms(V.vecchia_loglik_terms(p, yd, theta).cpu().numpy(), want[:, 0])
    tot = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    ref = oracle.compensated_sum(want)
    assert abs(tot[0] - ref[0]) <= W.LOGLIK_RTOL * np.abs(want[:, 0]).sum()
    for k in (1, 2, 3):
        assert abs(tot[k] - ref[k]) <= W.GRAD_RTOL * np.abs(want[:, k]).sum()
    if m == 150:  # m = n - 1 is exact: the Vecchia product is Eq. (1)
        xs = xy[:151]
        ys = y[:151]
        p2 = V.Plan(xs, 150)
        got = V.vecchia_loglik(p2, _dev(ys), theta).cpu().numpy()[0]
        assert abs(got - oracle.loglik_exact(xs, ys, theta)) <= 1e-9 * abs(got)
