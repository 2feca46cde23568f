"""Split-product oracle against exact rational arithmetic: digit ranges, the
reconstruction bound, exactness on small integers, and the truncation bound of
the kept slice pairs."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki


def test_digit_ranges_and_reconstruction():
    rng = np.random.default_rng(0)
    v = rng.standard_normal(300) * 10.0 ** rng.uniform(-8, 8, 300)
    E, D = ozaki.digits(v)
    assert np.all(np.abs(v) < 2.0 ** E)
    assert D[:, 0].min() >= -128 and D[:, 0].max() <= 128
    assert D[:, 1:].min() >= -128 and D[:, 1:].max() <= 128
    rec = ozaki.reconstruct(E, D)
    for a, r in zip(v, rec):
        # rounding after the sixth digit (weight 2^(E-47)): |a - rec| <= 2^(E-48)
        assert abs(Fraction(float(a)) - r) <= Fraction(2) ** (E - 48)


def test_zero_vector_and_sign():
    E, D = ozaki.digits(np.zeros(5))
    assert not D.any()
    E, D = ozaki.digits(np.array([-3.0, 3.0]))
    assert np.array_equal(D[0], -D[1])


def test_small_integers_are_one_digit():
    # max |v| = 127 gives E = 7, so the leading digit has weight 2^(E-7) = 1
    v = np.array([127.0, -127.0, 5.0, 0.0, -1.0])
    E, D = ozaki.digits(v)
    assert E == 7
    assert np.array_equal(D[:, 0], v.astype(np.int64)) and not D[:, 1:].any()
    # a vector holding 128 has E = 8: leading digits weigh 2, 128 -> 64
    E, D = ozaki.digits(np.array([128.0, 3.0]))
    assert E == 8 and D[0, 0] == 64 and D[1, 0] == 1 and D[1, 1] == 128


def test_integer_matrices_exact():
    rng = np.random.default_rng(1)
    L = rng.integers(-127, 128, (6, 40)).astype(float)
    R = rng.integers(-127, 128, (40, 5)).astype(float)
    assert np.array_equal(ozaki.split_product(L, R), L @ R)


@pytest.mark.parametrize("S", [4, 5, 6])
def test_truncation_bound(S):
    # the error of the split product is bounded by (i) rounding of each entry after
    # digit S and (ii) the dropped pairs: both <= K 2^(E_r+E_c) 2^(-8S+3)
    rng = np.random.default_rng(S)
    L = rng.standard_normal((4, 30))
    R = rng.standard_normal((30, 3))
    got = ozaki.split_product(L, R, S=S)
    ref = ozaki.exact_product(L, R)
    for i in range(4):
        for j in range(3):
            Er, Ec = ozaki.vector_exponent(L[i]), ozaki.vector_exponent(R[:, j])
            bound = 30 * 2.0 ** (Er + Ec) * 2.0 ** (-8 * S + 3)
            assert abs(got[i, j] - ref[i, j]) <= bound


def test_six_slices_reach_fp64_level():
    rng = np.random.default_rng(9)
    L = rng.standard_normal((10, 50))
    R = rng.standard_normal((50, 8))
    ref = ozaki.exact_product(L, R)
    err = np.linalg.norm(ozaki.split_product(L, R) - ref) / np.linalg.norm(ref)
    assert err < 1e-13
    err5 = np.linalg.norm(ozaki.split_product(L, R, S=5) - ref) / np.linalg.norm(ref)
    assert err5 > err   # one slice fewer loses ~8 bits


def test_subnormal_vector_is_sliced_exactly():
    # every entry subnormal: the vector still gets its own exponent (2^(E-1) <= max|a|
    # < 2^E) and, since subnormals are multiples of 2^-1074 and the last digit weighs
    # 2^(E-47) < 2^-1074 here, the six digits hold every entry exactly
    rng = np.random.default_rng(5)
    v = rng.standard_normal(64) * 2.0 ** -1040
    assert np.all((np.abs(v) < np.finfo(np.float64).tiny) & (v != 0))
    E, D = ozaki.digits(v)
    m = max(abs(Fraction(float(a))) for a in v)
    assert Fraction(2) ** (E - 1) <= m < Fraction(2) ** E
    assert ozaki.reconstruct(E, D) == [Fraction(float(a)) for a in v]
