"""The LDL^T pivot reciprocal (vecchia_pivot_reciprocal) against exact rational 1/d.

The kernels scale each eliminated column by 1/d_j computed without FP64 instructions
(FP32 seed, exact integer residual, second-order fixed-point correction).  Its claimed
accuracy, about half an ulp, is checked here against numpy's correctly rounded division
on a large sample and against exact fractions on a smaller one, with mantissas at the
edges of the seed's range (m = 1, just above 1, just below 2) and exponents across the
whole domain [2^-1022, 2^1022); values outside the domain give NaN.
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07412_gb300 import build, vecchia

    build.build()
    return vecchia


def _sample(n, seed):
    rng = np.random.default_rng(seed)
    frac = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    k = n // 8
    frac[:k] = rng.integers(0, 1 << 30, k, dtype=np.uint64)                    # m just above 1
    frac[k:2 * k] = (1 << 52) - 1 - rng.integers(0, 1 << 30, k, dtype=np.uint64)  # just below 2
    frac[2 * k:2 * k + 64] = 0                                                # m = 1
    expo = rng.integers(1, 2045, n, dtype=np.uint64)                          # whole domain
    expo[: n // 2] = rng.integers(1023 - 60, 1023 + 60, n // 2, dtype=np.uint64)
    return ((expo << np.uint64(52)) | frac).view(np.float64)


def _ulp(x):
    return np.spacing(np.abs(x))


def test_pivot_reciprocal_is_within_half_an_ulp(V):
    d = _sample(2_000_000, 7)
    got = V.vecchia_pivot_reciprocal(torch.as_tensor(d, device="cuda")).cpu().numpy()
    want = 1.0 / d  # correctly rounded
    assert np.all(np.isfinite(got))
    off = np.abs(got - want) / _ulp(want)
    assert off.max() <= 1.0, d[np.argmax(off)]
    assert np.mean(got == want) >= 0.99
    # exact error on a sub-sample, including every result that differs from numpy's
    idx = np.concatenate([np.flatnonzero(got != want)[:2000], np.arange(0, d.size, 997)])
    worst = 0.0
    for i in idx:
        exact = 1 / Fraction(float(d[i]))
        worst = max(worst, abs(float((Fraction(float(got[i])) - exact) / Fraction(float(_ulp(want[i]))))))
    assert worst <= 0.505, worst


def test_pivot_reciprocal_exact_cases_and_domain(V):
    inside = np.array([1.0, 2.0, 0.5, 3.0, 2.0 ** -1022, 2.0 ** 1021, np.nextafter(2.0 ** 1022, 0),
                       np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 1e-300, 1e300, 0.1, 7.0])
    got = V.vecchia_pivot_reciprocal(torch.as_tensor(inside, device="cuda")).cpu().numpy()
    want = 1.0 / inside
    assert np.all(np.abs(got - want) <= _ulp(want)), (inside, got, want)
    assert np.all(got[:6] == want[:6])  # powers of two and 3: exact or correctly rounded
    outside = np.array([0.0, -0.0, -1.0, 5e-324, 2.0 ** -1023, 2.0 ** 1022, 1e308, np.inf, -np.inf, np.nan])
    got = V.vecchia_pivot_reciprocal(torch.as_tensor(outside, device="cuda")).cpu().numpy()
    assert np.all(np.isnan(got)), got
    assert V.vecchia_pivot_reciprocal(torch.empty(0, dtype=torch.float64, device="cuda")).numel() == 0
