"""Pins of the oracle's emulated product (Section 2, Eq. 2 and threshold t).

* With every slice pair kept (t = 2s) the weighted level sums equal the exact
  integer product N_A N_B^T of the scaled integers (the closed form of Eq. 2).
* Small-integer matrices: the kept pairs already hold the whole product, so
  the emulated result equals the exact integer product.
* Entries with few significant bits: the kept sum is exact, so D equals the
  correctly rounded dot product (math.fsum of exact products).
* Random and log-scaled data: |D - AB| <= the a-priori bound, with AB exact.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import split, emulgemm, exact, bounds
from paper_2509_23565_gb300 import inputs


@pytest.mark.parametrize("s", [2, 3, 5, 7, 8])
def test_all_pairs_equal_integer_product(s):
    A = inputs.log_scaled(7, 9, 4, seed=11)
    B = inputs.log_scaled(9, 5, 4, seed=12)
    e, SA = split.split_rows(A, s)
    f, SB = split.split_cols(B, s)
    I = emulgemm.level_sums(SA, SB, 2 * s)
    T = emulgemm.combine_levels(I, 2 * s)
    NA = split.scaled_integers(A, e, s).astype(object)
    NB = split.scaled_integers(B.T, f, s).astype(object)
    want = NA.dot(NB.T)
    assert (T == want).all()


@pytest.mark.parametrize("s", [3, 4, 7, 8])
def test_small_integer_matrices_exact(s):
    rng = np.random.default_rng(20 + s)
    A = rng.integers(-100, 101, (13, 17)).astype(np.float64)
    B = rng.integers(-100, 101, (17, 6)).astype(np.float64)
    out = emulgemm.emul_gemm(A, B, s)
    want = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    assert (out == want).all()
    # C - AB in place form (alpha = -1, beta = 1)
    C = rng.integers(-1000, 1000, (13, 6)).astype(np.float64)
    out = emulgemm.emul_gemm(A, B, s, alpha=-1.0, beta=1.0, C=C)
    assert (out == C - want).all()


def test_correctly_rounded_dot_product():
    """Entries with at most 20 significant bits: every kept product is exact and
    no dropped pair is nonzero at s = 8, so D_ij = RN(sum_k a_ik b_kj)."""
    rng = np.random.default_rng(30)
    A = np.ldexp(rng.integers(-(2**20), 2**20, (5, 40)).astype(np.float64), -20)
    B = np.ldexp(rng.integers(-(2**20), 2**20, (40, 4)).astype(np.float64), -20)
    A[:, 0] = 0.999  # give every row a large entry so e_i is 0 for all rows
    A[:, 0] = np.ldexp(np.round(np.ldexp(A[:, 0], 20)), -20)
    B[0, :] = 1.0 - 2.0**-20
    out = emulgemm.emul_gemm(A, B, 8)
    for i in range(5):
        for j in range(4):
            want = math.fsum(float(A[i, k]) * float(B[k, j]) for k in range(40))
            assert out[i, j] == want


@pytest.mark.parametrize("s,r", [(3, 0), (5, 0), (6, 4), (7, 0), (7, 8), (8, 16)])
def test_error_within_a_priori_bound(s, r):
    A = inputs.log_scaled(6, 24, r, seed=40 + s) if r else inputs.uniform(6, 24, seed=40 + s)
    B = inputs.log_scaled(24, 5, r, seed=50 + s) if r else inputs.uniform(24, 5, seed=50 + s)
    D = emulgemm.emul_gemm(A, B, s)
    bnd = bounds.emul_bound(A, B, s, D)
    ex = exact.exact_product(A, B)
    for i in range(6):
        for j in range(5):
            err = abs(Fraction(float(D[i, j])) - ex[i][j])
            assert err <= Fraction(float(bnd[i, j])), (i, j, float(err), bnd[i, j])


def test_dropped_pairs_cost_at_most_bound_and_shrink():
    """Errors fall by roughly 2**7 per added slice (the per-slice factor behind Table 1)."""
    A = inputs.uniform(16, 128, seed=60)
    B = inputs.uniform(128, 16, seed=61)
    ex = np.array([[float(v) for v in row] for row in exact.exact_product(A, B)])
    errs = []
    for s in range(3, 8):
        D = emulgemm.emul_gemm(A, B, s)
        errs.append(np.abs(D - ex).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(30.0 < r < 1000.0 for r in ratios), ratios


def test_tolerance_against_fp64_where_slices_suffice():
    k = 256
    A = inputs.uniform(32, k, seed=70)
    B = inputs.uniform(k, 32, seed=71)
    fp64 = A @ B
    tol = 4 * k * 2.0**-53 * (np.abs(A) @ np.abs(B))
    for s in (7, 8):
        D = emulgemm.emul_gemm(A, B, s)
        mask = bounds.suffices(A, B, s, D)
        assert mask.mean() > 0.9
        assert (np.abs(D - fp64)[mask] <= tol[mask]).all()


def test_nonfinite_rows_give_nan():
    A = inputs.uniform(4, 8, seed=80)
    A[2, 3] = np.nan
    B = inputs.uniform(8, 3, seed=81)
    B[1, 2] = np.inf
    D = emulgemm.emul_gemm(A, B, 7)
    assert np.isnan(D[2]).all() and np.isnan(D[:, 2]).all()
    assert np.isfinite(np.delete(np.delete(D, 2, 0), 2, 1)).all()


def test_k_zero_and_beta_zero():
    A = np.zeros((3, 0))
    B = np.zeros((0, 4))
    C = np.ones((3, 4)) * 2.5
    out = emulgemm.emul_gemm(A, B, 7, alpha=-1.0, beta=1.0, C=C)
    assert (out == C).all()
    out = emulgemm.emul_gemm(A, B, 7)
    assert (out == 0).all()


@pytest.mark.parametrize("s", [2, 3, 4])
def test_threshold_full_product_correctly_rounded(s):
    """Threshold t = 2s keeps every slice pair: with entries of at most 7s
    significant bits below their row's (column's) scale nothing is truncated by
    the split, so D_ij = RN(sum_k a_ik b_kj).  The method's t = s + 1 drops
    the pairs with p + q > s + 1, which are nonzero here, and must differ."""
    rng = np.random.default_rng(70 + s)
    bits = 7 * s - 1
    A = np.ldexp(rng.integers(-(2**bits), 2**bits, (6, 30)).astype(np.float64), -bits)
    B = np.ldexp(rng.integers(-(2**bits), 2**bits, (30, 5)).astype(np.float64), -bits)
    A[:, 0] = 0.5 + 2.0**-bits       # row scales 2^0
    B[0, :] = -(0.5 + 2.0**-bits)    # column scales 2^0
    ex = exact.exact_product(A, B)
    want = np.array([[float(ex[i][j]) for j in range(5)] for i in range(6)])   # Fraction -> nearest double
    assert np.array_equal(emulgemm.emul_gemm(A, B, s, t=2 * s), want)
    assert not np.array_equal(emulgemm.emul_gemm(A, B, s), want)
    # every intermediate threshold lies between: error non-increasing in t
    errs = [float(np.max(np.abs(emulgemm.emul_gemm(A, B, s, t=t) - want))) for t in range(2, 2 * s + 1)]
    assert all(a >= b for a, b in zip(errs, errs[1:])) and errs[-1] == 0.0, errs


@pytest.mark.parametrize("s,sa", [(7, 3), (8, 5), (6, 6), (5, 1)])
def test_shorter_split_is_a_prefix(s, sa):
    """The slices of an sa-slice split are the leading sa slices of an s-slice
    split (same scales): truncation at 7 sa bits keeps the leading digits."""
    A = inputs.log_scaled(9, 33, 6, seed=40 + s)
    e, S = split.split_rows(A, s)
    e2, S2 = split.split_rows(A, sa)
    assert np.array_equal(e, e2)
    assert np.array_equal(S[:sa], S2)


@pytest.mark.parametrize("sa,sb", [(3, 7), (7, 4), (5, 5), (2, 8), (8, 1)])
def test_unequal_all_pairs_equal_truncated_product(sa, sb):
    """With t = sa + sb every pair p <= sa, q <= sb is kept, and the kept sum
    T = sum_{p,q} SA_p SB_q 2^(7(t-p-q)) is exactly N_A^(sa) N_B^(sb)^T, the
    product of the scaled integers truncated to 7 sa and 7 sb bits."""
    A = inputs.log_scaled(6, 11, 3, seed=50 + sa)
    B = inputs.log_scaled(11, 5, 3, seed=60 + sb)
    s = max(sa, sb)
    t = sa + sb
    e, SA = split.split_rows(A, s)
    f, SB = split.split_cols(B, s)
    T = emulgemm.combine_levels(emulgemm.level_sums(SA, SB, t, sa=sa, sb=sb), t)
    NA = split.scaled_integers(A, e, sa).astype(object)
    NB = split.scaled_integers(B.T, f, sb).astype(object)
    assert (T == NA.dot(NB.T)).all()
    # and the rounded result is RN of that exact product times 2^(e + f - 7 (sa + sb))
    D = emulgemm.emul_gemm_unequal(A, B, sa, sb, t=t)
    for i in range(6):
        for j in range(5):
            want = Fraction(int(NA[i].dot(NB[j]))) * Fraction(2) ** (int(e[i]) + int(f[j]) - 7 * t)
            assert D[i, j] == float(want)


def test_unequal_equal_counts_is_the_method():
    A = inputs.uniform(20, 30, seed=70)
    B = inputs.uniform(30, 9, seed=71)
    for s in (3, 7):
        assert np.array_equal(emulgemm.emul_gemm_unequal(A, B, s, s), emulgemm.emul_gemm(A, B, s))


def test_unequal_fewer_slices_never_more_accurate():
    """Dropping slices of one operand can only lose digits: with t = sa + sb
    the error against the exact product grows as sa shrinks."""
    A = inputs.uniform(30, 64, seed=72)
    B = inputs.uniform(64, 20, seed=73)
    ref = np.array([[float(sum(Fraction(A[i, k]) * Fraction(B[k, j]) for k in range(64))) for j in range(20)]
                    for i in range(30)])
    errs = []
    for sa in (2, 4, 6, 8):
        D = emulgemm.emul_gemm_unequal(A, B, sa, 8, t=sa + 8)
        errs.append(np.abs(D - ref).max())
    assert all(errs[i] > errs[i + 1] for i in range(3)), errs
