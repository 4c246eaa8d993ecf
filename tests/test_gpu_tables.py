"""The per-smoothness covariance table cache under pressure.

Each nu gets a table built on the GPU the first time it is used; the cache holds a
bounded number and rebuilds the least recently used one in place when it is full,
ordered after every earlier reader on any stream (no device-wide synchronisation, no
free).  Here 70 distinct nu values cycle through the cache twice, in opposite orders,
and calls alternate between two streams: every result must be bit-identical to its
first evaluation, and a few must match the oracle.
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


def test_many_nu_values_cycle_through_the_cache(V):
    n, m = 6000, 12
    xy = datagen.uniform_locations(n, 301)
    y = datagen.field_rff(xy, (1.0, 0.05, 1.0, 0.02), 302, features=512)
    p = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=303)
    yd = torch.as_tensor(y, device="cuda")
    nus = [0.31 + 0.047 * k for k in range(70)]
    first = {}
    for nu in nus:
        first[nu] = V.vecchia_loglik_grad(p, yd, (1.1, 0.04, nu, 0.02)).cpu().numpy()
    # a plan serves one stream at a time: the second stream gets its own (identical) plan
    q = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=303)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    outs = []
    for k, nu in enumerate(reversed(nus)):
        st, pl = (s1, p) if k % 2 == 0 else (s2, q)
        with torch.cuda.stream(st):
            o = torch.empty(4, dtype=torch.float64, device="cuda")
            V.vecchia_loglik_grad(pl, yd, (1.1, 0.04, nu, 0.02), out=o)
            outs.append((nu, o))
    torch.cuda.synchronize()
    q.close()
    for nu, o in outs:
        assert np.array_equal(o.cpu().numpy(), first[nu]), nu
    perm = p.perm()
    for nu in (nus[0], nus[33], nus[69]):
        th = (1.1, 0.04, nu, 0.02)
        want = oracle.vecchia_rows(xy[perm], y[perm], m, th)
        assert abs(first[nu][0] - oracle.compensated_sum(want)[0]) <= W.LOGLIK_RTOL * np.abs(want).sum()
    # the covariance evaluator shares the cache
    d = torch.linspace(0.0, 0.3, 1000, dtype=torch.float64, device="cuda")
    for nu in (nus[5], nus[60]):
        c = V.vecchia_matern(d, (1.0, 0.04, nu, 0.0), with_dbeta=False).cpu().numpy()
        ref = oracle.matern(d.cpu().numpy(), 1.0, 0.04, nu)
        assert np.all(np.abs(c - ref) <= 4e-15)
    p.close()
