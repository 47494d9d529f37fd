"""Pins of the oracle's scale extraction and slicing (Section 2, Eq. 1-4).

Each check compares the oracle with something other than itself: exact integer
/ Fraction arithmetic on the IEEE-754 values, the closed-form digit identity,
and the range example of Eq. 3.
"""
import math
import sys
from fractions import Fraction

import numpy as np
import pytest

from oracle import split
from paper_2509_23565_gb300 import inputs


def _smallest_e_bruteforce(x):
    """Smallest integer e with |x| < 2**e, from the exact ratio of x."""
    x = abs(float(x))
    p, q = x.as_integer_ratio()          # q is a power of two
    e = p.bit_length() - q.bit_length() + 1
    assert Fraction(x) < Fraction(2) ** e and not Fraction(x) < Fraction(2) ** (e - 1)
    return e


def _special_values():
    tiny = 5e-324
    return np.array([1.0, -1.0, 0.5, 0.75, 2.0**-1022, tiny, 3 * tiny, -2.0**-1074 * 12345,
                     sys.float_info.max, -sys.float_info.max, 1.0 - 2**-53, 2.0**52 + 1, -3.0,
                     1e300, -1e-300, 2.0**-1023, 7.0 * 2**-1060])


def test_row_exponents_match_bruteforce():
    rng = np.random.default_rng(1)
    vals = np.concatenate([_special_values(), rng.standard_normal(40) * 10.0 ** rng.integers(-300, 300, 40)])
    A = vals.reshape(-1, 1) * np.array([[1.0, 0.25, -0.5]])
    e = split.row_exponents(A)
    for i in range(A.shape[0]):
        assert e[i] == _smallest_e_bruteforce(np.abs(A[i]).max())


def test_zero_and_nonfinite_rows():
    A = np.array([[0.0, -0.0, 0.0], [1.0, np.inf, 2.0], [np.nan, 1.0, 1.0], [0.0, 3.0, 0.0]])
    e = split.row_exponents(A)
    assert e[0] == 0
    assert e[1] == split.NONFINITE and e[2] == split.NONFINITE
    assert e[3] == 2
    N = split.scaled_integers(A, e, 7)
    assert (N[:3] == 0).all()


@pytest.mark.parametrize("s", [3, 5, 7, 8])
def test_scaled_integers_are_truncations(s):
    rng = np.random.default_rng(2 + s)
    A = np.concatenate([_special_values().reshape(-1, 1) * rng.uniform(-1, 1, (1, 6)),
                        inputs.log_scaled(12, 6, 16, seed=3)], axis=0)
    A[0, 0] = 0.0
    e = split.row_exponents(A)
    N = split.scaled_integers(A, e, s)
    W = 7 * s
    for i in range(A.shape[0]):
        for k in range(A.shape[1]):
            want = int(Fraction(float(A[i, k])) * Fraction(2) ** (W - int(e[i])))   # int() truncates toward 0
            assert int(N[i, k]) == want
            assert abs(want) < 2**W


@pytest.mark.parametrize("s", [1, 2, 3, 7, 8])
def test_digits_recompose_and_range(s):
    rng = np.random.default_rng(10 + s)
    A = inputs.uniform(9, 11, seed=4) * 10.0 ** rng.integers(-5, 5, (9, 1))
    e, S = split.split_rows(A, s)
    N = split.scaled_integers(A, e, s)
    assert S.dtype == np.int8 and S.shape == (s, 9, 11)
    assert np.abs(S.astype(np.int64)).max() <= 127
    recomposed = np.zeros_like(N)
    for p in range(1, s + 1):
        recomposed = recomposed * 128 + S[p - 1].astype(np.int64)
    assert (recomposed == N).all()
    # every digit carries the sign of its entry
    sgn = np.sign(A)[None].repeat(s, 0)
    assert (S.astype(np.int64) * sgn >= 0).all()


def test_reconstruction_exact_when_wide_enough():
    """With E_ij the smallest E with |a_ij| < 2**E, the slices reconstruct a_ij
    exactly when W >= 53 + (e_i - E_ij) (all significand bits lie within W)."""
    s = 8
    W = 7 * s
    A = inputs.uniform(6, 20, seed=5)
    e, S = split.split_rows(A, s)
    rec = split.reconstruct(S, e)
    checked = 0
    for i in range(6):
        for k in range(20):
            Eik = _smallest_e_bruteforce(A[i, k]) if A[i, k] != 0 else -10**9
            if W >= 53 + (int(e[i]) - Eik):
                assert rec[i][k] == Fraction(float(A[i, k]))
                checked += 1
            else:
                assert abs(rec[i][k] - Fraction(float(A[i, k]))) < Fraction(2) ** (int(e[i]) - W)
    assert checked > 60


def test_range_example_eq3():
    """Eq. 3: rows 2**53 and 2**-53 times the identity.  A single scale for the
    whole of A rounds the second row to 0; per-row scales keep it exactly."""
    from oracle import emulgemm
    A = np.array([[2.0**53, 2.0**53], [2.0**-53, 2.0**-53]])
    B = np.eye(2)
    s = 7
    out = emulgemm.emul_gemm(A, B, s)
    assert (out == A).all()
    # shared scale: use the largest row exponent for every row
    e = split.row_exponents(A)
    shared = np.full_like(e, e.max())
    N = split.scaled_integers(A, shared, s)
    assert (N[1] == 0).all() and (N[0] != 0).all()
