"""Exact reference products (pins for the emulated product of Section 2).

Every FP64 number is a dyadic rational, so sum_k a_ik b_kj is computed exactly
with Python Fractions.  Used on small matrices and sampled entries only.

Test infrastructure only (see the package docstring).
"""
from fractions import Fraction

import numpy as np


def exact_entry(A, B, i, j):
    """Exact sum_k A[i,k] * B[k,j] as a Fraction."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    return sum((Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(A.shape[1])),
               Fraction(0))


def exact_product(A, B):
    """Exact A @ B as a nested list of Fractions."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    Af = [[Fraction(float(x)) for x in row] for row in A]
    Bf = [[Fraction(float(x)) for x in row] for row in B]
    m, k = A.shape
    n = B.shape[1]
    return [[sum((Af[i][kk] * Bf[kk][j] for kk in range(k)), Fraction(0)) for j in range(n)]
            for i in range(m)]


def abs_product(A, B):
    """(|A| |B|) in float64 (the scale of the componentwise error bound)."""
    return np.abs(np.asarray(A, dtype=np.float64)) @ np.abs(np.asarray(B, dtype=np.float64))
