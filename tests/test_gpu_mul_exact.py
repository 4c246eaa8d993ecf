"""The integer column-scaling product (vecchia_mul_by_positive) against IEEE FP64 products.

The full-warp kernels scale each eliminated column by its pivot reciprocal with an
integer product of the two 53-bit mantissas, rounded to nearest even, so that no FP64
instruction sits on the column step's serial path.  The claim is bit-identity with the
FP64 multiply wherever the exact product is finite and at least 2^-1022 in magnitude.
numpy's float64 multiply (IEEE round to nearest, ties to even) is the reference: two
million random operand pairs over wide exponent ranges, then the edges — mantissa
carries into the exponent, exact ties, the smallest and largest normal results, and
zero or subnormal left operands.
"""
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


def _bits(x):
    return np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)


def _from_bits(sign, expo, frac):
    return ((np.uint64(sign) << np.uint64(63)) | (np.asarray(expo, dtype=np.uint64) << np.uint64(52))
            | np.asarray(frac, dtype=np.uint64)).view(np.float64)


def _run(V, a, b):
    ad = torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    bd = torch.as_tensor(np.ascontiguousarray(b), device="cuda")
    return V.vecchia_mul_by_positive(ad, bd).cpu().numpy()


def _scaled(a, b):
    # |a| b 2^600 rounded once in the normal range: strictly above 2^-422 means the exact
    # product is above 2^-1022, strictly below means it is below (rounding is monotonic
    # and 2^-422 is a double); equality is left out of both sets.
    with np.errstate(over="ignore"):
        return (np.abs(a) * 2.0 ** 600) * b


def _assert_matches_ieee(got, a, b):
    with np.errstate(over="ignore", under="ignore"):
        want = a * b
    normal = np.isfinite(want) & (_scaled(a, b) > 2.0 ** -422)
    bad = np.flatnonzero(normal & (_bits(got) != _bits(want)))
    assert bad.size == 0, (bad[:5], a[bad[:5]], b[bad[:5]], got[bad[:5]], want[bad[:5]])
    over = np.isinf(want)
    assert np.array_equal(got[over], want[over])
    # exact products below 2^-1022 give a zero of a's sign
    tiny = _scaled(a, b) < 2.0 ** -422
    assert np.all(got[tiny] == 0.0) and np.array_equal(np.signbit(got[tiny]), np.signbit(a[tiny]))
    return normal, tiny


def test_random_products_bit_identical(V):
    rng = np.random.default_rng(2024)
    n = 2_000_000
    # a: signed, mantissas uniform, exponents mostly moderate (the kernels' column entries),
    # a quarter across the whole normal range; b: positive normal, likewise
    ea = rng.integers(1023 - 80, 1023 + 80, n)
    ea[: n // 4] = rng.integers(1, 2047, n // 4)
    eb = rng.integers(1023 - 80, 1023 + 80, n)
    eb[n // 4: n // 2] = rng.integers(1, 2047, n // 4)
    a = _from_bits(0, ea, rng.integers(0, 1 << 52, n, dtype=np.uint64))
    a[rng.random(n) < 0.5] *= -1.0
    b = _from_bits(0, eb, rng.integers(0, 1 << 52, n, dtype=np.uint64))
    got = _run(V, a, b)
    normal, tiny = _assert_matches_ieee(got, a, b)
    assert normal.sum() > 1_500_000 and tiny.sum() > 1000


def test_carries_ties_and_range_edges(V):
    rng = np.random.default_rng(7)
    k = np.arange(1, 20001, dtype=np.uint64)
    cases_a, cases_b = [], []
    # ties: (1 + k 2^-52)(1 + 2^-1) = 1.5 + 1.5 k 2^-52, a half-ulp remainder for odd k
    cases_a.append(_from_bits(0, 1023, k))
    cases_b.append(np.full(k.size, 1.5))
    # ties at the [2, 4) binade: (1 + k 2^-52)(1 + 2^-1 + 2^-2) products cross 2
    cases_a.append(_from_bits(0, 1023, (1 << 52) - k))
    cases_b.append(np.full(k.size, 1.75))
    # mantissa carries: all-ones mantissas times values just above 1
    ones = np.full(k.size, (1 << 52) - 1, dtype=np.uint64)
    cases_a.append(_from_bits(0, rng.integers(900, 1100, k.size), ones))
    cases_b.append(_from_bits(0, 1023, k))
    cases_a.append(_from_bits(1, rng.integers(900, 1100, k.size), ones - (k & np.uint64(7))))
    cases_b.append(_from_bits(0, 1023, (k & np.uint64(3))))
    # results at the bottom of the normal range: exact products at or just above 2^-1022
    cases_a.append(_from_bits(0, 1, rng.integers(0, 1 << 52, k.size, dtype=np.uint64)))
    cases_b.append(_from_bits(0, 1023, rng.integers(0, 1 << 10, k.size, dtype=np.uint64)))
    cases_a.append(np.full(k.size, 2.0 ** -511))
    cases_b.append(_from_bits(0, 1023 - 511, rng.integers(0, 1 << 52, k.size, dtype=np.uint64)))
    # exact products just below 2^-1022, which IEEE rounding may lift to 2^-1022: zero here
    cases_a.append(_from_bits(0, 1, (1 << 52) - 1 - (k & np.uint64(15))))
    cases_b.append(np.full(k.size, 0.5))
    # results at the top: up to the largest double, and beyond it (infinity)
    cases_a.append(_from_bits(0, 2046, rng.integers(0, 1 << 52, k.size, dtype=np.uint64)))
    cases_b.append(_from_bits(0, 1022, rng.integers(0, 1 << 52, k.size, dtype=np.uint64)))
    cases_a.append(_from_bits(0, 2046, ones))
    cases_b.append(_from_bits(0, 1023, k))
    a = np.concatenate(cases_a)
    b = np.concatenate(cases_b)
    got = _run(V, a, b)
    normal, tiny = _assert_matches_ieee(got, a, b)
    assert normal.sum() > 6 * k.size and tiny.sum() >= k.size
    with np.errstate(over="ignore"):
        assert np.isinf(a * b).sum() > 1000
    # zero and subnormal left operands give a zero of their sign
    z = np.array([0.0, -0.0, 5e-324, -5e-324, 2.0 ** -1030, -(2.0 ** -1023)])
    gz = _run(V, z, np.full(z.size, 3.0))
    assert np.all(gz == 0.0) and np.array_equal(np.signbit(gz), np.signbit(z))
