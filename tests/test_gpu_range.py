"""The location-range call (vecchia_loglik_range), the deterministic reduction, and the
error slot's failure kinds.

The likelihood is a sum of n independent terms (Sec. V-B); the range call evaluates a
contiguous range of ordered locations, the unit by which the multi-GPU path splits a
field.  k = 2, 3 and 7 disjoint ranges (shard.location_ranges, the split that path
uses), summed on the host in rank order, must equal the unsplit call within the
likelihood tolerances, for the warp kernels and the CTA kernel.  Two identical calls
must give identical bits.  A non-finite y makes the result NaN and is reported at the
first ordered location whose block holds it, with status EINVAL.
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


def _field(n, m, seed, theta, order=1):
    from paper_2403_07412_gb300 import vecchia as V

    xy = datagen.gmm_locations(n, seed) if order == 2 else datagen.uniform_locations(n, seed)
    y = datagen.field_rff(xy, theta, seed + 1, features=512)
    return xy, y, V.Plan(xy, m, order=order, seed=seed + 2)


@pytest.mark.parametrize("n,m,order", [(30_000, 60, 2), (20_000, 30, 1), (12_000, 10, 1), (3000, 90, 1)])
def test_disjoint_ranges_sum_to_the_unsplit_call(V, n, m, order):
    from paper_2403_07412_gb300 import shard

    theta = (1.1, 0.04, 1.0, 0.02)
    xy, y, p = _field(n, m, 60 + m, theta, order)
    yd = _dev(y)
    full = V.vecchia_loglik_grad(p, yd, theta).cpu().numpy()
    full_fwd = V.vecchia_loglik(p, yd, theta).cpu().numpy()
    terms = V.vecchia_loglik_terms(p, yd, theta, want_grad=True).cpu().numpy()
    den = np.abs(terms).sum(axis=0)
    # the whole range is the unsplit call itself: same launch, same records, same bits
    assert np.array_equal(V.vecchia_loglik_range(p, yd, theta, 0, n, want_grad=True).cpu().numpy(), full)
    assert np.array_equal(V.vecchia_loglik_range(p, yd, theta, 0, n).cpu().numpy(), full_fwd)
    for k in (2, 3, 7):
        parts = [V.vecchia_loglik_range(p, yd, theta, i0, i1, want_grad=True).cpu().numpy()
                 for i0, i1 in shard.location_ranges(n, k)]
        summed = [math.fsum(pt[c] for pt in parts) for c in range(4)]
        assert abs(summed[0] - full[0]) <= W.LOGLIK_RTOL * den[0], (k, summed[0], full[0])
        for c in (1, 2, 3):
            assert abs(summed[c] - full[c]) <= W.GRAD_RTOL * den[c], (k, c, summed[c], full[c])
        # each range against the sum of its own terms
        for (i0, i1), pt in zip(shard.location_ranges(n, k), parts):
            seg = terms[i0:i1]
            assert abs(pt[0] - seg[:, 0].sum()) <= W.LOGLIK_RTOL * den[0]
        fparts = [V.vecchia_loglik_range(p, yd, theta, i0, i1).cpu().numpy()[0]
                  for i0, i1 in shard.location_ranges(n, k)]
        assert abs(math.fsum(fparts) - full_fwd[0]) <= W.LOGLIK_RTOL * den[0]
    p.close()


def test_range_edges_and_rejections(V):
    theta = (1.0, 0.05, 1.5, 0.01)
    xy, y, p = _field(5000, 20, 71, theta)
    yd = _dev(y)
    z = V.vecchia_loglik_range(p, yd, theta, 1234, 1234, want_grad=True).cpu().numpy()
    assert np.array_equal(z, np.zeros(4))
    # a single location, and the first one (no conditioning set): l_0 = log N(y; 0, sigma2 + tau2)
    terms = V.vecchia_loglik_terms(p, yd, theta).cpu().numpy()
    one = V.vecchia_loglik_range(p, yd, theta, 777, 778).cpu().numpy()[0]
    assert abs(one - terms[777]) <= 1e-12 * max(1.0, abs(terms[777]))
    y0 = y[p.perm()[0]]
    first = V.vecchia_loglik_range(p, yd, theta, 0, 1).cpu().numpy()[0]
    v = theta[0] + theta[3]
    assert abs(first - (-0.5 * y0 * y0 / v - 0.5 * math.log(v) - 0.5 * math.log(2 * math.pi))) < 1e-14
    for i0, i1 in ((-1, 10), (10, 9), (0, 5001), (4999, 5002)):
        with pytest.raises(V.VecchiaError) as e:
            V.vecchia_loglik_range(p, yd, theta, i0, i1)
        assert e.value.code == V.EINVAL
    p.close()


@pytest.mark.parametrize("m", [10, 30, 60, 100])
def test_repeated_calls_are_bit_identical(V, m):
    theta = (1.3, 0.05, 1.0, 0.03)
    xy, y, p = _field(40_000 if m <= 63 else 4000, m, 80 + m, theta)
    yd = _dev(y)
    for fn in (V.vecchia_loglik, V.vecchia_loglik_grad):
        a = fn(p, yd, theta).cpu().numpy()
        b = fn(p, yd, theta).cpu().numpy()
        assert np.array_equal(a, b) and np.all(np.isfinite(a))
    p.close()


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_nonfinite_y_reported_at_its_location(V, bad):
    theta = (1.0, 0.08, 0.5, 0.01)
    n, m = 3000, 15
    xy, y, p = _field(n, m, 91, theta)
    perm = p.perm()
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    orig = int(perm[1717])
    yb = y.copy()
    yb[orig] = bad
    yd = _dev(yb)
    for fn in (V.vecchia_loglik, V.vecchia_loglik_grad):
        out = fn(p, yd, theta).cpu().numpy()
        assert np.isnan(out[0])
        # conditioning sets hold earlier points only, so the first block holding y[orig]
        # is that location's own
        assert p.last_error() == (1717, V.EINVAL)
    # clean data clears the slot
    ok = V.vecchia_loglik(p, _dev(y), theta).cpu().numpy()
    assert np.isfinite(ok[0]) and p.last_error() == (-1, V.OK)
    # a range that excludes the location is unaffected
    r = V.vecchia_loglik_range(p, yd, theta, 0, 1717).cpu().numpy()
    assert np.isfinite(r[0]) and p.last_error() == (-1, V.OK)
    p.close()


def test_not_positive_definite_status_is_enotpd(V):
    xy = datagen.uniform_locations(200, 14)
    perm = oracle.order_random(200, 15)
    xy[perm[57]] = xy[perm[3]]          # duplicate of an earlier point, no nugget
    p = V.Plan(xy, 8, order=V.ORDER_GIVEN, perm=perm)
    y = _dev(np.linspace(-1, 1, 200))
    out = V.vecchia_loglik_grad(p, y, (1.0, 0.1, 0.5, 0.0)).cpu().numpy()
    assert np.all(np.isnan(out[[0, 1, 2, 3]]))
    assert p.last_error() == (57, V.ENOTPD)
    p.close()
