"""A-priori error bound of the emulated product (Section 2 of arXiv 2509.23565).

The paper states that dropping the slice-pair products with i+j > t is the
only rounding of the scheme and leaves the analysis out of scope.  Bound used
here, with s slices of 7 bits, W = 7s, t = s+1 and scaled entries
alpha_ik = a_ik 2**-e_i, beta_kj = b_kj 2**-f_j (|alpha|, |beta| < 1):

* input truncation: alpha = N 2**-W + d with |d| < 2**-W, so each of the k
  products carries at most 2*2**-W + 2**-2W;
* dropped levels L = s+2..2s: at most (2s+1-L) pairs of |S| <= 127 < 2**7,
  sum_L (2s+1-L) 2**(14-7L) < 1.01 (s-1) 2**-7s per product;
* the single rounding of the kept sum: at most u |D| (u = 2**-53).

    |D_ij - (AB)_ij| <= 2**(e_i+f_j) * k * (s + 1.02) * 2**(-7s) + u |D_ij|

The slice count "suffices" for entry (i,j) when this bound is at most
3 k u (|A||B|)_ij, so that together with the error k u (|A||B|)_ij of a plain
FP64 product the emulated entry lies within 4 k u (|A||B|)_ij of it.

Test infrastructure only (see the package docstring).
"""
import numpy as np

from .split import NONFINITE, row_exponents, col_exponents

U = 2.0 ** -53


def emul_bound(A, B, s, D=None):
    """Entrywise a-priori bound on |D - AB| (float64 [m, n])."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    k = A.shape[1]
    e = row_exponents(A).astype(np.float64)
    f = col_exponents(B).astype(np.float64)
    e[e == NONFINITE] = np.inf
    f[f == NONFINITE] = np.inf
    scale = np.exp2(e[:, None] + f[None, :])
    b = scale * k * (s + 1.02) * 2.0 ** (-7 * s)
    if D is not None:
        b = b + U * np.abs(D)
    return b


def suffices(A, B, s, D=None):
    """Boolean mask of entries where s slices meet the 4 k u (|A||B|) tolerance."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    k = A.shape[1]
    absprod = np.abs(A) @ np.abs(B)
    return emul_bound(A, B, s, D) <= 3.0 * k * U * absprod
