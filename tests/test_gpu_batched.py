"""GPU tests of the batched many-field, many-theta persistent launch."""
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


def _fields(V, sizes, ms, seed, given_perm=False):
    plans, ys, hosts = [], [], []
    for f, (n, m) in enumerate(zip(sizes, ms)):
        xy = datagen.uniform_locations(n, seed + f)
        th0 = (1.0, 0.05, 1.0, 0.02)
        y = datagen.field_rff(xy, th0, seed + 100 + f, features=512)
        if given_perm:
            perm = oracle.order_random(n, seed + 200 + f)
            p = V.Plan(xy, m, order=V.ORDER_GIVEN, perm=perm)
        else:
            p = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=seed + 300 + f)
        plans.append(p)
        ys.append(torch.as_tensor(y, device="cuda"))
        hosts.append((xy, y))
    return plans, ys, hosts


def test_batched_matches_single_field_calls(V):
    sizes = [3000, 8000, 20_000, 1500, 12_000, 5000]
    ms = [10, 30, 60, 10, 30, 60]
    plans, ys, _ = _fields(V, sizes, ms, 1000)
    nth = 4
    thetas = datagen.theta_candidates(len(sizes), nth, 7)
    V.vecchia_batched_prepare([0.5, 1.0, 1.5])
    b = V.Batch(plans, ys, nth, want_grad=True)
    td = torch.as_tensor(thetas, device="cuda").contiguous()
    out = b.run(td).cpu().numpy()
    for f in range(len(sizes)):
        for t in range(nth):
            th = thetas[f, t]
            ref = V.vecchia_loglik_grad(plans[f], ys[f], th).cpu().numpy()
            terms = V.vecchia_loglik_terms(plans[f], ys[f], th, want_grad=True).cpu().numpy()
            den = np.abs(terms).sum(axis=0)
            assert abs(out[f, t, 0] - ref[0]) <= W.LOGLIK_RTOL * den[0], (f, t)
            for k in (1, 2, 3):
                assert abs(out[f, t, k] - ref[k]) <= W.GRAD_RTOL * den[k], (f, t, k)
    # forward only
    bf = V.Batch(plans, ys, nth, want_grad=False)
    outf = bf.run(td).cpu().numpy()
    np.testing.assert_allclose(outf[..., 0], out[..., 0], rtol=1e-12, atol=0)


def test_batched_against_oracle(V):
    sizes, ms = [1200, 2000, 900], [10, 30, 60]
    plans, ys, hosts = _fields(V, sizes, ms, 2000, given_perm=True)
    nth = 3
    thetas = datagen.theta_candidates(len(sizes), nth, 11)
    V.vecchia_batched_prepare([0.5, 1.0, 1.5])
    out = V.Batch(plans, ys, nth).run(torch.as_tensor(thetas, device="cuda").contiguous()).cpu().numpy()
    for f, (n, m) in enumerate(zip(sizes, ms)):
        xy, y = hosts[f]
        perm = oracle.order_random(n, 2000 + 200 + f)
        for t in range(nth):
            terms = oracle.vecchia_rows(xy[perm], y[perm], m, thetas[f, t], want_grad=True)
            want = oracle.compensated_sum(terms)
            den = np.abs(terms).sum(axis=0)
            assert abs(out[f, t, 0] - want[0]) <= W.LOGLIK_RTOL * den[0]
            for k in (1, 2, 3):
                assert abs(out[f, t, k] - want[k]) <= W.GRAD_RTOL * den[k], (f, t, k)


def test_batched_graph_capture_and_replay(V):
    sizes, ms = [4000, 2500, 6000], [30, 10, 60]
    plans, ys, _ = _fields(V, sizes, ms, 3000)
    nth = 5
    V.vecchia_batched_prepare([0.5, 1.0, 1.5])
    b = V.Batch(plans, ys, nth, want_grad=True)
    th_a = torch.as_tensor(datagen.theta_candidates(3, nth, 21), device="cuda").contiguous()
    th_b = torch.as_tensor(datagen.theta_candidates(3, nth, 22), device="cuda").contiguous()
    static_th = th_a.clone()
    static_out = torch.empty((3, nth, 4), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(static_th, static_out)  # lays out the work before capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run(static_th, static_out)
    for th in (th_b, th_a):
        static_th.copy_(th)
        g.replay()
        torch.cuda.synchronize()
        direct = b.run(th).cpu().numpy()
        np.testing.assert_array_equal(static_out.cpu().numpy(), direct)


def test_batched_unprepared_nu_gives_nan(V):
    plans, ys, _ = _fields(V, [2000, 3000], [10, 30], 4000)
    V.vecchia_batched_prepare([0.5])
    th = np.array([[[1.0, 0.05, 0.5, 0.01]], [[1.0, 0.05, 2.5, 0.01]]])
    out = V.Batch(plans, ys, 1).run(torch.as_tensor(th, device="cuda").contiguous()).cpu().numpy()
    assert np.all(np.isfinite(out[0])) and np.all(np.isnan(out[1]))
    ref = V.vecchia_loglik_grad(plans[0], ys[0], th[0, 0]).cpu().numpy()
    assert abs(out[0, 0, 0] - ref[0]) <= 1e-9 * abs(ref[0])
