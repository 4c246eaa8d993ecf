"""Parity on the timed configuration itself: n = 1,000,000 locations from the
20-component Gaussian mixture, maxmin ordering, m = 60, Matérn nu = 1 (the workload
bench.py times), plus the 250k-location differentiation workload at its stated size.

The ordering is checked bit for bit against the oracle's O(n^2) greedy maxmin: in full at
250k clustered locations, and on the first 20,000 picks of the 1M plan.  On the 1M plan,
sampled ordered rows (the first ones, the m / m + 1 boundary and 300 from every decile of
the ordering) must have the oracle's brute-force conditioning sets bit for bit, and
their log-likelihood terms and gradients must match the oracle's (1e-9 and 1e-7).
"""
import numpy as np
import pytest
import torch

import oracle
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


@pytest.fixture(scope="module")
def scale_plan(V):
    xy, y, theta, m, order = W.scale(device="cuda")
    assert order == W.ORDER_MAXMIN and xy.shape[0] == 1_000_000 and m == 60
    plan = V.Plan(xy, m, order=V.ORDER_MAXMIN)
    yield xy, y, theta, m, plan
    plan.close()


def _sample_rows(n, m, per_decile=300, seed=11):
    rng = np.random.default_rng(seed)
    rows = [np.array([0, 1, 2, m - 1, m, m + 1, m + 2])]
    edges = np.linspace(0, n, 11).astype(np.int64)
    for a, b in zip(edges[:-1], edges[1:]):
        rows.append(rng.choice(np.arange(a, b), per_decile, replace=False))
    rows.append(np.array([n - 1]))
    return np.unique(np.concatenate(rows))


def _check(got, want):
    err = np.abs(got[:, 0] - want[:, 0])
    bad = np.flatnonzero(err > W.LOGLIK_RTOL * np.maximum(np.abs(want[:, 0]), 1.0))
    assert bad.size == 0, (bad[:5], got[bad[:5], 0], want[bad[:5], 0])
    scale = np.abs(want[:, 1:]).mean(axis=0)
    gerr = np.abs(got[:, 1:] - want[:, 1:])
    bad = np.argwhere(gerr > W.GRAD_RTOL * np.maximum(np.abs(want[:, 1:]), scale))
    assert bad.size == 0, (bad[:5], got[bad[:5, 0]], want[bad[:5, 0]])


def test_maxmin_ordering_bit_exact_250k_clustered(V):
    xy, _, _, m, _ = W.scale(n=250_000)
    p = V.Plan(xy, m, order=V.ORDER_MAXMIN)
    np.testing.assert_array_equal(p.perm(), oracle.order_maxmin(xy))
    p.close()


def test_timed_plan_ordering_prefix_bit_exact(scale_plan):
    xy, _, _, _, plan = scale_plan
    perm = plan.perm()
    assert np.array_equal(np.sort(perm), np.arange(xy.shape[0]))
    np.testing.assert_array_equal(perm[:20_000], oracle.order_maxmin_prefix(xy, 20_000))


def test_timed_plan_neighbors_terms_and_gradients(V, scale_plan):
    xy, y, theta, m, plan = scale_plan
    n = xy.shape[0]
    perm = plan.perm()
    xo, yo = xy[perm], y[perm]
    rows = _sample_rows(n, m)
    assert rows.size >= 3000
    want_nbr = oracle.knn_rows(xo, m, rows)
    np.testing.assert_array_equal(plan.neighbors()[rows], want_nbr)
    yd = torch.as_tensor(y, device="cuda")
    terms = V.vecchia_loglik_terms(plan, yd, theta, want_grad=True).cpu().numpy()
    want = oracle.vecchia_rows(xo, yo, m, theta, rows=rows, nbr=want_nbr, want_grad=True)
    _check(terms[rows], want)
    # the forward-only kernel gives the same terms as the gradient kernel's first column
    fwd = V.vecchia_loglik_terms(plan, yd, theta).cpu().numpy()
    _check(np.column_stack([fwd[rows], want[:, 1:]]), want)
    # totals of the timed call are the sums of the terms
    tot = V.vecchia_loglik_grad(plan, yd, theta).cpu().numpy()
    den = np.abs(terms).sum(axis=0)
    assert abs(tot[0] - terms[:, 0].sum()) <= W.LOGLIK_RTOL * den[0]
    for k in (1, 2, 3):
        assert abs(tot[k] - terms[:, k].sum()) <= W.GRAD_RTOL * den[k]


def test_differentiation_workload_central_differences_250k(V):
    # The adjoint against central finite differences of the forward kernel, h = 1e-6
    # relative, on the 250k-location differentiation workload (random ordering, m = 60,
    # nu = 2.5).
    xy, y, theta, m, order = W.differentiation()
    assert xy.shape[0] == 250_000 and m == 60
    p = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=3)
    yd = torch.as_tensor(y, device="cuda")
    g = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    for k, ti in ((1, 0), (2, 1), (3, 3)):
        h = 1e-6 * theta[ti]
        tp, tm = list(theta), list(theta)
        tp[ti] += h
        tm[ti] -= h
        fd = (float(V.vecchia_loglik(p, yd, tp).cpu()[0]) - float(V.vecchia_loglik(p, yd, tm).cpu()[0])) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(g[0]), (k, g[k], fd)
    p.close()
