"""Pins for the CPU oracle: each test ties it to something other than itself.

Sources of truth used here: closed forms of Eq. (2) at half-integer nu, scipy's
independent Bessel-K (AMOS) and multivariate normal log-density, the values of
Table II, published splitmix64 outputs, brute force on tiny inputs, and exact
identities of the Vecchia construction (Sec. V-B): m = n-1 reproduces Eq. (1),
the sigma^2 scaling law, and the KL ordering of Eq. (5).
"""
import math
import os

import numpy as np
import pytest
from scipy.special import gamma as sp_gamma, kv
from scipy.stats import multivariate_normal, norm

from paper_2403_07412_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


# ----------------------------------------------------------------- Eq. (2)
@pytest.mark.parametrize("nu,closed", [
    (0.5, lambda x: np.exp(-x)),
    (1.5, lambda x: (1 + x) * np.exp(-x)),
    (2.5, lambda x: (1 + x + x * x / 3) * np.exp(-x)),
])
def test_matern_half_integer_closed_forms(oracle_mod, nu, closed):
    # With Eq. (2)'s parametrisation (no sqrt(2 nu)), K_{n+1/2} gives e^{-x} times a polynomial.
    d = np.concatenate([np.linspace(1e-6, 0.05, 50), np.linspace(0.05, 3.0, 200)])
    beta, sigma2 = 0.07, 1.7
    got = oracle_mod.matern(d, sigma2, beta, nu)
    want = sigma2 * closed(d / beta)
    np.testing.assert_allclose(got, want, rtol=2e-14, atol=1e-300)
    assert oracle_mod.matern([0.0], sigma2, beta, nu)[0] == sigma2


@pytest.mark.parametrize("nu", [0.3, 0.5, 1.0, 1.7, 2.5, 3.2])
def test_bessel_k_against_scipy(oracle_mod, nu):
    x = np.geomspace(1e-6, 200.0, 400)
    np.testing.assert_allclose(oracle_mod.bessel_k(x, nu), kv(nu, x), rtol=5e-13)


def test_bessel_k_half_order_closed_form(oracle_mod):
    x = np.geomspace(1e-4, 300.0, 300)
    np.testing.assert_allclose(oracle_mod.bessel_k(x, 0.5), np.sqrt(np.pi / (2 * x)) * np.exp(-x),
                               rtol=1e-14)


def test_matern_general_nu_against_scipy(oracle_mod):
    d = np.geomspace(1e-7, 2.0, 300)
    for nu in (0.8, 1.0, 2.2):
        want = 2 ** (1 - nu) / sp_gamma(nu) * (d / 0.03) ** nu * kv(nu, d / 0.03)
        np.testing.assert_allclose(oracle_mod.matern(d, 1.0, 0.03, nu), want, rtol=1e-12, atol=1e-300)


def test_table2_effective_range_invariant(oracle_mod):
    # Table II: every (nu, beta) pair puts the same correlation level at its effective range.
    rows = np.loadtxt(os.path.join(GOLDEN, "table2_beta.txt"))
    vals = np.array([oracle_mod.matern([r], 1.0, b, nu)[0] for nu, r, b in rows])
    assert np.all(np.abs(vals - 0.022222) < 3e-6), vals


def test_matern_dbeta_finite_difference(oracle_mod):
    d = np.geomspace(1e-4, 0.5, 60)
    for nu in (0.5, 1.0, 2.5, 0.7):
        beta, h = 0.05, 1e-6 * 0.05
        fd = (oracle_mod.matern(d, 1.3, beta + h, nu) - oracle_mod.matern(d, 1.3, beta - h, nu)) / (2 * h)
        np.testing.assert_allclose(oracle_mod.matern_dbeta(d, 1.3, beta, nu), fd, rtol=2e-7, atol=2e-8)
    assert oracle_mod.matern_dbeta([0.0], 1.0, 0.1, 1.0)[0] == 0.0


def test_powexp_closed_form_and_matern_identity(oracle_mod):
    # Eq. (3) with exponent 1 is Eq. (2) with nu = 1/2 (both sigma2 exp(-d/beta)).
    d = np.geomspace(1e-6, 3.0, 300)
    np.testing.assert_allclose(oracle_mod.powexp(d, 1.4, 0.08, 1.0), oracle_mod.matern(d, 1.4, 0.08, 0.5),
                               rtol=2e-14)
    for a in (0.5, 1.5, 2.0):
        np.testing.assert_allclose(oracle_mod.powexp(d, 0.9, 0.2, a), 0.9 * np.exp(-d ** a / 0.2), rtol=1e-13)
        h = 1e-6 * 0.2
        fd = (oracle_mod.powexp(d, 0.9, 0.2 + h, a) - oracle_mod.powexp(d, 0.9, 0.2 - h, a)) / (2 * h)
        np.testing.assert_allclose(oracle_mod.powexp_dbeta(d, 0.9, 0.2, a), fd, rtol=1e-6, atol=1e-9)


def test_powexp_exact_and_vecchia_full_conditioning(oracle_mod):
    n = 80
    theta = (1.3, 0.05, 1.5, 0.02)
    xy = datagen.uniform_locations(n, 91)
    dd = np.sqrt(((xy[:, None] - xy[None]) ** 2).sum(-1))
    S = theta[0] * np.exp(-dd ** theta[2] / theta[1]) + theta[3] * np.eye(n)
    y = np.linalg.cholesky(S) @ np.random.default_rng(1).standard_normal(n)
    want = multivariate_normal(mean=np.zeros(n), cov=S).logpdf(y)
    ex, gex = oracle_mod.loglik_exact(xy, y, theta, want_grad=True, family=1)
    assert _rel(ex, want) < 1e-10
    va = oracle_mod.vecchia(xy, y, n - 1, theta, want_grad=True, family=1)
    assert _rel(va[0], ex) < 1e-10
    np.testing.assert_allclose(va[1:], gex, rtol=1e-8, atol=1e-8 * np.abs(gex).max())


# ----------------------------------------------------------------- orderings
def test_splitmix64_published_vector(oracle_mod):
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    assert [int(v) for v in oracle_mod.splitmix64(0, 3)] == want


def test_order_random_small_case_by_hand(oracle_mod):
    # Durstenfeld shuffle driven by the published outputs, done by hand for n = 4.
    outs = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    a = [0, 1, 2, 3]
    for step, i in enumerate((3, 2, 1)):
        j = outs[step] % (i + 1)
        a[i], a[j] = a[j], a[i]
    assert oracle_mod.order_random(4, 0).tolist() == a


def test_order_random_is_uniform(oracle_mod):
    # A uniform shuffle leaves the last element in place with probability 1/n
    # (Sattolo's variant never does) and puts each element in each slot equally often.
    n, trials = 6, 6000
    counts = np.zeros((n, n))
    for s in range(trials):
        p = oracle_mod.order_random(n, 1000 + s)
        assert sorted(p.tolist()) == list(range(n))
        counts[p, np.arange(n)] += 1
    expected = trials / n
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 60.0, chi2  # 25 dof; p ~ 1e-4
    assert counts.min() > 0


def _maxmin_brute(xy):
    n = len(xy)
    c = xy.mean(axis=0)
    d0 = ((xy - c) ** 2).sum(1)
    order = [int(np.argmin(d0))]
    mind = np.full(n, np.inf)
    used = np.zeros(n, bool)
    used[order[0]] = True
    for _ in range(n - 1):
        last = xy[order[-1]]
        mind = np.minimum(mind, ((xy - last) ** 2).sum(1))
        cand = np.where(~used, mind, -1.0)
        j = int(np.flatnonzero(cand == cand.max())[0])
        order.append(j)
        used[j] = True
    return np.array(order)


def test_order_maxmin_matches_brute_force(oracle_mod):
    for seed in range(3):
        xy = datagen.uniform_locations(300, seed)
        np.testing.assert_array_equal(oracle_mod.order_maxmin(xy), _maxmin_brute(xy))


def test_order_maxmin_prefix_is_the_leading_part(oracle_mod):
    # The stopped-early form takes the same greedy steps: its output is the first
    # `count` entries of numpy brute force (and of the full ordering).
    xy = datagen.gmm_locations(500, 9)
    full = _maxmin_brute(xy)
    for count in (1, 2, 37, 500):
        np.testing.assert_array_equal(oracle_mod.order_maxmin_prefix(xy, count), full[:count])
    np.testing.assert_array_equal(oracle_mod.order_maxmin(xy), full)
    with pytest.raises(ValueError):
        oracle_mod.order_maxmin_prefix(xy, 501)


def test_order_maxmin_grid_structure(oracle_mod):
    # 3x3 grid: start at the centre; then the four corners (each at squared distance
    # 0.5 from the centre, ties to the lowest index), then the edge midpoints.
    g = np.array([[x, y] for y in (0.0, 0.5, 1.0) for x in (0.0, 0.5, 1.0)])
    p = oracle_mod.order_maxmin(g)
    assert p[:5].tolist() == [4, 0, 2, 6, 8]
    assert sorted(p.tolist()) == list(range(9))


def test_order_maxmin_property(oracle_mod):
    # Each chosen point has the largest distance to the already chosen set.
    xy = datagen.gmm_locations(400, 7)
    p = oracle_mod.order_maxmin(xy)
    pts = xy[p]
    for k in range(1, 400):
        dk = ((pts[k:, None, :] - pts[None, :k, :]) ** 2).sum(-1).min(1)
        assert dk[0] == dk.max()


def test_order_morton_z_pattern(oracle_mod):
    # 4x4 grid (x fastest): the Z-order visits 2x2 quads in Z order, each quad in Z order.
    g = np.array([[x, y] for y in (0.0, 1 / 3, 2 / 3, 1.0) for x in (0.0, 1 / 3, 2 / 3, 1.0)])
    want = [0, 1, 4, 5, 2, 3, 6, 7, 8, 9, 12, 13, 10, 11, 14, 15]
    assert oracle_mod.order_morton(g).tolist() == want
    # duplicates keep their original order; a degenerate (constant) axis maps to cell 0
    pts = np.array([[0.5, 0.2], [0.5, 0.9], [0.5, 0.2], [0.5, 0.0]])
    assert oracle_mod.order_morton(pts).tolist() == [3, 0, 2, 1]


def test_order_morton_matches_sorting_by_interleaved_key(oracle_mod):
    xy = datagen.gmm_locations(3000, 9)
    lo, hi = xy.min(0), xy.max(0)
    q = np.minimum(np.floor((xy - lo) / (hi - lo) * 65536.0), 65535).astype(np.int64)
    key = np.zeros(len(xy), dtype=np.int64)
    for b in range(16):
        key |= ((q[:, 0] >> b) & 1) << (2 * b)
        key |= ((q[:, 1] >> b) & 1) << (2 * b + 1)
    np.testing.assert_array_equal(oracle_mod.order_morton(xy), np.lexsort((np.arange(len(xy)), key)))


# ----------------------------------------------------------------- kNN
def test_knn_against_numpy_brute_force(oracle_mod):
    xy = datagen.uniform_locations(700, 3)
    xy[5] = xy[2]            # duplicate point: distance ties broken by index
    xy[40] = xy[11]
    m = 12
    got = oracle_mod.knn_rows(xy, m)
    for i in range(700):
        want = np.full(m, -1)
        if i:
            d = (xy[:i, 0] - xy[i, 0]) ** 2 + (xy[:i, 1] - xy[i, 1]) ** 2
            o = np.lexsort((np.arange(i), d))[:m]
            want[:o.size] = o
        np.testing.assert_array_equal(got[i], want)


def test_knn_rows_subset_matches_full(oracle_mod):
    xy = datagen.uniform_locations(500, 4)
    full = oracle_mod.knn_rows(xy, 7)
    rows = np.array([0, 1, 7, 8, 250, 499])
    np.testing.assert_array_equal(oracle_mod.knn_rows(xy, 7, rows), full[rows])


# ----------------------------------------------------------------- Eq. (1)
def _cov_scipy(xy, theta):
    s2, b, nu, t2 = theta
    d = np.sqrt(((xy[:, None] - xy[None]) ** 2).sum(-1))
    with np.errstate(invalid="ignore"):
        C = s2 * 2 ** (1 - nu) / sp_gamma(nu) * (d / b) ** nu * kv(nu, d / b)
    C[d == 0] = s2
    return C + t2 * np.eye(len(xy))


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5, 0.0), (1.5, 0.05, 1.0, 0.05), (0.7, 0.2, 2.5, 0.01)])
def test_exact_loglik_against_scipy(oracle_mod, theta):
    xy = datagen.uniform_locations(120, 11)
    y = datagen.field_dense(xy, theta, 12)
    want = multivariate_normal(mean=np.zeros(120), cov=_cov_scipy(xy, theta)).logpdf(y)
    assert _rel(oracle_mod.loglik_exact(xy, y, theta), want) < 1e-10


# ----------------------------------------------------------------- Vecchia
@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5, 0.0), (1.5, 0.03, 2.5, 0.05), (1.0, 0.05, 1.0, 0.01)])
def test_vecchia_full_conditioning_equals_exact(oracle_mod, theta):
    # With m = n-1 every conditional is exact, so the Vecchia product is Eq. (1).
    n = 90
    xy = datagen.uniform_locations(n, 21)
    y = datagen.field_dense(xy, theta, 22)
    perm = oracle_mod.order_random(n, 5)
    xo, yo = xy[perm], y[perm]
    va = oracle_mod.vecchia(xo, yo, n - 1, theta, want_grad=True)
    ex, gex = oracle_mod.loglik_exact(xy, y, theta, want_grad=True)
    assert _rel(va[0], ex) < 1e-10
    np.testing.assert_allclose(va[1:], gex, rtol=1e-8, atol=1e-8 * np.abs(gex).max())


def test_first_terms_closed_form(oracle_mod):
    # l_1 = log N(y_1; 0, sigma2 + tau2); l_2 conditions on one point.
    theta = (1.3, 0.08, 1.5, 0.02)
    xy = datagen.uniform_locations(5, 1)
    y = np.array([0.4, -0.9, 0.1, 0.3, 0.2])
    t = oracle_mod.vecchia_rows(xy, y, 3, theta)
    v = theta[0] + theta[3]
    assert _rel(t[0], norm.logpdf(y[0], 0, math.sqrt(v))) < 1e-14
    c = oracle_mod.matern([math.dist(xy[0], xy[1])], theta[0], theta[1], theta[2])[0]
    mu, s = c / v * y[0], v - c * c / v
    assert _rel(t[1], norm.logpdf(y[1], mu, math.sqrt(s))) < 1e-13


def test_sigma2_scaling_identity(oracle_mod):
    # tau2 = 0: Sigma(sigma2) = sigma2 Sigma(1), so mu_i is unchanged, s_i scales by sigma2 and
    # l(sigma2) = l(1) - n/2 log sigma2 - (1/sigma2 - 1) Q1/2, Q1 = sum r_i^2 / s_i at sigma2 = 1.
    n, m = 400, 10
    xy = datagen.uniform_locations(n, 31)
    y = datagen.field_dense(xy, (1.0, 0.1, 1.0, 0.0), 32)
    t1, ms = oracle_mod.vecchia_rows(xy, y, m, (1.0, 0.1, 1.0, 0.0), return_mu_s=True)
    q1 = float((((y - ms[:, 0]) ** 2) / ms[:, 1]).sum())
    for s2 in (0.3, 2.7):
        l = oracle_mod.vecchia(xy, y, m, (s2, 0.1, 1.0, 0.0), want_grad=True)
        want = t1.sum() - n / 2 * math.log(s2) - (1 / s2 - 1) * q1 / 2
        assert _rel(l[0], want) < 1e-12
        assert _rel(l[1], -n / (2 * s2) + q1 / (2 * s2 * s2)) < 1e-9


def test_kl_ordering_eq5(oracle_mod):
    # Eq. (5) with y = 0: D_KL = l0 - la >= 0, and la grows with m (nested conditioning sets).
    n = 150
    theta = (1.0, 0.1, 1.5, 0.0)
    xy = datagen.uniform_locations(n, 41)
    xo = xy[oracle_mod.order_random(n, 9)]
    y0 = np.zeros(n)
    l0 = oracle_mod.loglik_exact(xo, y0, theta)
    prev = -np.inf
    for m in (1, 3, 10, 30, 80, n - 1):
        la = oracle_mod.vecchia(xo, y0, m, theta)
        assert la <= l0 + 1e-9 * abs(l0)
        assert la >= prev - 1e-9 * abs(l0)
        prev = la
    assert _rel(prev, l0) < 1e-10


def test_block_logdensity_matches_scipy(oracle_mod):
    # log N(y; 0, S) of one dense block against scipy's multivariate normal: a wrong
    # log-determinant factor, a transposed solve or a dropped 2 pi term would fail here.
    rng = np.random.default_rng(12)
    for k in (1, 2, 5, 17, 40):
        A = rng.standard_normal((k, k))
        S = A @ A.T + 0.3 * k * np.eye(k)
        y = 2.0 * rng.standard_normal(k)
        want = multivariate_normal(mean=np.zeros(k), cov=S).logpdf(y)
        assert _rel(oracle_mod.block_logdensity(S, y), want) < 1e-12, k
    with pytest.raises(oracle_mod.OracleNotPD):
        oracle_mod.block_logdensity(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2))


def test_identity_padding_leaves_block_density(oracle_mod):
    # Sec. V-B pads short sets with dummy vectors; identity rows with y = 0 add log N(0;0,1) each.
    rng = np.random.default_rng(0)
    A = rng.standard_normal((6, 6))
    S = A @ A.T + 6 * np.eye(6)
    y = rng.standard_normal(6)
    P = np.eye(9)
    P[3:, 3:] = S
    yp = np.concatenate([np.zeros(3), y])
    base = oracle_mod.block_logdensity(S, y)
    assert _rel(oracle_mod.block_logdensity(P, yp) - 3 * norm.logpdf(0.0), base) < 1e-13


@pytest.mark.parametrize("theta", [(1.5, 0.03, 2.5, 0.05), (1.0, 0.1, 0.5, 0.02), (1.0, 0.02, 1.0, 0.01)])
def test_vecchia_gradient_central_differences(oracle_mod, theta):
    n, m = 300, 15
    xy = datagen.uniform_locations(n, 51)
    y = datagen.field_rff(xy, theta, 52, features=512)
    g = oracle_mod.vecchia(xy, y, m, theta, want_grad=True)
    for k, ti in ((1, 0), (2, 1), (3, 3)):
        h = 1e-6 * theta[ti]
        tp, tm = list(theta), list(theta)
        tp[ti] += h
        tm[ti] -= h
        fd = (oracle_mod.vecchia(xy, y, m, tp) - oracle_mod.vecchia(xy, y, m, tm)) / (2 * h)
        assert _rel(g[k], fd) < 2e-6, (k, g[k], fd)


def test_not_positive_definite_is_reported(oracle_mod):
    xy = np.array([[0.1, 0.1], [0.1, 0.1], [0.5, 0.5]])
    y = np.array([0.1, 0.2, 0.3])
    with pytest.raises(oracle_mod.OracleNotPD) as e:
        oracle_mod.vecchia_rows(xy, y, 2, (1.0, 0.1, 0.5, 0.0))
    assert e.value.row == 1


# ----------------------------------------------------------------- Sec. VI-C: sphere
R_EARTH = 6371.0


def test_gcd_special_values(oracle_mod):
    a = np.array([[0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [10.0, 20.0], [-75.0, 40.0], [30.0, 89.0]])
    b = np.array([[0.0, 90.0], [180.0, 0.0], [1.0, 0.0], [10.0, 20.0], [-75.0, 41.0], [210.0, 89.0]])
    got = oracle_mod.gcd(a, b, R_EARTH)
    want = R_EARTH * np.radians([90.0, 180.0, 1.0, 0.0, 1.0, 2.0])  # meridian arcs and the pole
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-9)
    np.testing.assert_allclose(oracle_mod.gcd(b, a, R_EARTH), got, rtol=0, atol=0)


def test_gcd_matches_chord_of_unit_vectors(oracle_mod):
    # d = 2 r asin(|u - v| / 2): an independent formula on numpy unit vectors.
    g = datagen.rng(41)
    a = np.stack([g.uniform(-180, 180, 2000), np.degrees(np.arcsin(g.uniform(-1, 1, 2000)))], 1)
    b = a + g.normal(scale=[5.0, 3.0], size=a.shape)
    b[:, 1] = np.clip(b[:, 1], -90, 90)
    ua, ub = datagen.sphere_coords(a, 1.0), datagen.sphere_coords(b, 1.0)
    want = 2.0 * R_EARTH * np.arcsin(np.linalg.norm(ua - ub, axis=1) / 2.0)
    np.testing.assert_allclose(oracle_mod.gcd(a, b, R_EARTH), want, rtol=1e-11, atol=1e-9)
    xyz = oracle_mod.sphere_xyz(a)
    np.testing.assert_allclose(np.linalg.norm(xyz, axis=1), 1.0, rtol=1e-15)
    np.testing.assert_allclose(xyz, ua, atol=1e-15)


def test_knn_sphere_against_numpy_great_circle(oracle_mod):
    ll = datagen.sphere_locations(3000, 42)
    xyz = oracle_mod.sphere_xyz(ll)
    rows = np.array([1, 5, 17, 200, 999, 2999])
    got = oracle_mod.knn_rows_sphere(xyz, 12, rows)
    u = datagen.sphere_coords(ll, 1.0)
    for r, row in zip(rows, got):
        d = 2.0 * np.arcsin(np.linalg.norm(u[:r] - u[r], axis=1) / 2.0)  # great-circle angle
        want = np.lexsort((np.arange(r), d))[:min(r, 12)]
        assert list(row[:min(r, 12)]) == list(want)
        assert np.all(row[min(r, 12):] == -1)


@pytest.mark.parametrize("family,theta", [(0, (1.0, 150.0, 0.5, 0.0)), (0, (1.3, 80.0, 0.5, 0.02)),
                                          (1, (1.0, 30.0, 0.8, 0.01))])
def test_sphere_full_conditioning_equals_dense(oracle_mod, family, theta):
    # m = n-1 Vecchia = Eq. (1) with great-circle distances; the dense likelihood itself
    # is checked against scipy with a covariance built from numpy's chord formula.
    n = 80
    ll = datagen.sphere_locations(n, 43)
    u = datagen.sphere_coords(ll, 1.0)
    d = 2.0 * R_EARTH * np.arcsin(np.clip(np.linalg.norm(u[:, None] - u[None], axis=-1) / 2.0, 0, 1))
    s2, b, nu, t2 = theta
    if family == 0:
        C = oracle_mod.matern(d.ravel(), s2, b, nu).reshape(n, n)
    else:
        C = s2 * np.exp(-d ** nu / b)
    S = C + t2 * np.eye(n) + (0.0 if t2 > 0 else 1e-10) * np.eye(n)
    y = np.linalg.cholesky(S) @ datagen.rng(44).standard_normal(n)
    ex, gex = oracle_mod.loglik_exact(ll, y, theta, want_grad=True, family=family, radius=R_EARTH)
    if t2 > 0:
        want = multivariate_normal(mean=np.zeros(n), cov=C + t2 * np.eye(n)).logpdf(y)
        assert _rel(ex, want) < 1e-9
    perm = oracle_mod.order_random(n, 6)
    va = oracle_mod.vecchia(ll[perm], y[perm], n - 1, theta, want_grad=True, family=family, radius=R_EARTH)
    assert _rel(va[0], ex) < 1e-10
    np.testing.assert_allclose(va[1:], gex, rtol=1e-8, atol=1e-8 * np.abs(gex).max())



# ----------------------------------------------------------------- prediction (kriging)
def test_predict_interpolates_observed_points(oracle_mod):
    # tau2 = 0: at an observed location the conditional mean is y there and the variance 0.
    xy = datagen.uniform_locations(400, 51)
    theta = (1.3, 0.1, 1.5, 0.0)
    y = datagen.field_dense(xy, theta, 52)
    mean, var, nbr = oracle_mod.predict(xy, y, xy[:40], 12, theta)
    np.testing.assert_allclose(mean, y[:40], rtol=0, atol=1e-12)
    assert np.all(np.abs(var) <= 1e-12)
    assert np.all(nbr[:, 0] == np.arange(40))


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5, 0.05), (1.5, 0.06, 2.5, 0.01)])
def test_predict_with_all_points_is_dense_kriging(oracle_mod, theta):
    n, k = 150, 30
    xy = datagen.uniform_locations(n + k, 53)
    y = datagen.field_dense(xy[:n], theta, 54)
    mean, var, _ = oracle_mod.predict(xy[:n], y, xy[n:], n, theta)
    S = _cov_scipy(xy[:n], theta)
    s2, b, nu, t2 = theta
    d = np.sqrt(((xy[n:, None] - xy[None, :n]) ** 2).sum(-1))
    Kx = s2 * 2 ** (1 - nu) / sp_gamma(nu) * (d / b) ** nu * kv(nu, d / b)
    want_mean = Kx @ np.linalg.solve(S, y)
    want_var = s2 + t2 - np.einsum("ij,ji->i", Kx, np.linalg.solve(S, Kx.T))
    np.testing.assert_allclose(mean, want_mean, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(var, want_var, rtol=1e-8, atol=1e-11)


def test_predict_neighbours_brute_force(oracle_mod):
    xy = datagen.uniform_locations(2000, 55)
    new = datagen.uniform_locations(50, 56)
    _, _, nbr = oracle_mod.predict(xy, np.zeros(2000), new, 15, (1.0, 0.1, 0.5, 0.01))
    for k in range(50):
        dx, dy = xy[:, 0] - new[k, 0], xy[:, 1] - new[k, 1]
        d2 = dx * dx + dy * dy
        assert list(nbr[k]) == list(np.lexsort((np.arange(2000), d2))[:15])


def test_predict_on_sphere_is_dense_kriging(oracle_mod):
    n, k = 120, 20
    ll = datagen.sphere_locations(n + k, 57)
    theta = (1.0, 70.0, 0.5, 0.02)
    u = datagen.sphere_coords(ll, 1.0)
    d = 2.0 * R_EARTH * np.arcsin(np.clip(np.linalg.norm(u[:, None] - u[None], axis=-1) / 2.0, 0, 1))
    C = theta[0] * np.exp(-d / theta[1])  # nu = 1/2: the exponential
    y = np.linalg.cholesky(C[:n, :n] + theta[3] * np.eye(n)) @ datagen.rng(58).standard_normal(n)
    mean, var, _ = oracle_mod.predict(ll[:n], y, ll[n:], n, theta, radius=R_EARTH)
    S = C[:n, :n] + theta[3] * np.eye(n)
    Kx = C[n:, :n]
    np.testing.assert_allclose(mean, Kx @ np.linalg.solve(S, y), rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(var, theta[0] + theta[3] - np.einsum("ij,ji->i", Kx, np.linalg.solve(S, Kx.T)),
                               rtol=1e-8, atol=1e-11)
