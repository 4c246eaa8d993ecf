"""The allocation-free log-likelihood entry point (vecchia_loglik_noalloc).

It serves callers that may not allocate device memory; its scratch is a fixed
device array inside the library.  Its index arrays come from the caller, so the kernel
checks them before reading through them: an entry outside [0, n) gives NaN, not an
out-of-bounds read.  This file sorts last so that a run stopping at the
first failure has already run every other test; it passes alone in a fresh process
too (the first call on the device performs the scratch look-up).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2403_07412_gb300 import datagen
from tests import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07412_gb300 import build, vecchia as V

    build.build()
    n, m = 20_000, 30
    theta = (1.2, 0.04, 1.0, 0.02)
    xy = datagen.gmm_locations(n, 31)
    y = datagen.field_rff(xy, theta, 32, features=1024)
    plan = V.Plan(xy, m, order=V.ORDER_MAXMIN)
    perm = plan.perm()
    nbr = plan.neighbors()
    nbr_orig = np.where(nbr >= 0, perm[np.maximum(nbr, 0)], -1).astype(np.int32)
    dev = torch.device("cuda")
    xy_d = torch.as_tensor(np.ascontiguousarray(xy), device=dev)
    y_d = torch.as_tensor(y, device=dev)
    nbr_d = torch.as_tensor(nbr_orig, device=dev)
    self_d = torch.as_tensor(perm.astype(np.int32), device=dev)
    want = V.vecchia_loglik(plan, y_d, theta).cpu().numpy()[0]
    terms = V.vecchia_loglik_terms(plan, y_d, theta).cpu().numpy()
    tol = W.LOGLIK_RTOL * np.abs(terms).sum()
    L = V.lib()
    th = (ctypes.c_double * 4)(*theta)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        rc = L.vecchia_loglik_noalloc(ctypes.c_void_p(xy_d.data_ptr()), ctypes.c_void_p(y_d.data_ptr()),
                                      ctypes.c_void_p(nbr_d.data_ptr()), ctypes.c_void_p(self_d.data_ptr()),
                                      n, m, th, ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == V.OK
        got = out.cpu().numpy()[0]
        assert abs(got - want) <= tol, (got, want)
    # arguments outside the limits are rejected before any device work
    assert L.vecchia_loglik_noalloc(ctypes.c_void_p(xy_d.data_ptr()), ctypes.c_void_p(y_d.data_ptr()),
                                    ctypes.c_void_p(nbr_d.data_ptr()), ctypes.c_void_p(self_d.data_ptr()),
                                    n, V.MAX_M_WARP + 1, th, ctypes.c_void_p(out.data_ptr()), stream) == V.EINVAL


def test_noalloc_out_of_range_indices_give_nan():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07412_gb300 import build, vecchia as V

    build.build()
    n, m = 4000, 20
    theta = (1.0, 0.06, 1.5, 0.02)
    xy = datagen.uniform_locations(n, 41)
    y = datagen.field_rff(xy, theta, 42, features=256)
    plan = V.Plan(xy, m, order=V.ORDER_RANDOM, seed=43)
    perm = plan.perm()
    nbr = plan.neighbors()
    nbr_orig = np.where(nbr >= 0, perm[np.maximum(nbr, 0)], -1).astype(np.int32)
    dev = torch.device("cuda")
    xy_d = torch.as_tensor(np.ascontiguousarray(xy), device=dev)
    y_d = torch.as_tensor(y, device=dev)
    self_ok = perm.astype(np.int32)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    want = V.vecchia_loglik(plan, y_d, theta).cpu().numpy()[0]
    cases = []
    for row, slot, val in ((2500, 7, n), (2500, 0, -1), (5, 4, 2 ** 31 - 1)):  # slot 4 < m_5 = 5
        bad = nbr_orig.copy()
        bad[row, slot] = val
        cases.append((bad, self_ok))
    bad_self = self_ok.copy()
    bad_self[999] = -7
    cases.append((nbr_orig, bad_self))
    for nb, sf in cases:
        V.vecchia_loglik_noalloc(xy_d, y_d, torch.as_tensor(nb, device=dev), torch.as_tensor(sf, device=dev), m,
                                 theta, out)
        assert np.isnan(out.cpu().numpy()[0])
    # padding beyond m_i is never read: a garbage pad does not matter
    pad = nbr_orig.copy()
    pad[3, 10:] = 123456789
    V.vecchia_loglik_noalloc(xy_d, y_d, torch.as_tensor(pad, device=dev), torch.as_tensor(self_ok, device=dev), m,
                             theta, out)
    got = out.cpu().numpy()[0]
    terms = V.vecchia_loglik_terms(plan, y_d, theta).cpu().numpy()
    assert abs(got - want) <= W.LOGLIK_RTOL * np.abs(terms).sum(), (got, want)
