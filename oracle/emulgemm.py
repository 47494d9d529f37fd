"""Emulated DGEMM by slice-pair products: Section 2, Eq. 1-2 and the truncation
threshold t of arXiv 2509.23565; used as the Schur-complement update of Eq. 7.

With a_ik ~ 2**e_i sum_p SA_p(i,k) 2**(-7p) and b_kj ~ 2**f_j sum_q SB_q(j,k) 2**(-7q):

    (AB)_ij ~ 2**(e_i+f_j) * sum_{L=2..t} 2**(-7L) * I_L(i,j),
    I_L = sum_{p+q=L} SA_p SB_q^T          (exact integers, "level sums")

Products with p+q > t are dropped; the paper calls this the only rounding of
the scheme.  Reading: t = s+1 (so s(s+1)/2 slice-pair products).

Recombination reading (the paper is silent): the kept levels are summed
exactly, T = sum_L I_L 2**(7(t-L)), and rounded once to FP64:
    D_ij = RN(T_ij * 2**(e_i + f_j - 7t)).
The C update is then the plain IEEE FP64 one, out = RN(RN(alpha*D) + RN(beta*C))
(beta = 0: out = RN(alpha*D), C not read).  For the Schur update of Eq. 7
(alpha = -1, beta = 1) that is out = RN(C - D).  A row/column with a NONFINITE
scale gives NaN in its products.

Test infrastructure only (see the package docstring).
"""
import math
import numpy as np

from .split import BITS, NONFINITE, split_rows, split_cols


def level_sums(SA, SB, t, sa=None, sb=None):
    """I[L-2] = sum_{p+q=L} SA[p-1] @ SB[q-1]^T for L = 2..t, as int64 [t-1, m, n].

    SA: int8 [s, m, k]; SB: int8 [s, n, k].  With sa / sb given only the pairs
    with p <= sa and q <= sb are summed (unequal slice counts, see
    emul_gemm_unequal).  Each product term is at most 127**2 and each partial
    sum at most k * s * 127**2 < 2**53 for the sizes used here, so float64
    matmul of the integer-valued planes is exact in any summation order; the
    result is converted back to int64.
    """
    s = SA.shape[0]
    sa = s if sa is None else sa
    sb = s if sb is None else sb
    m, k = SA.shape[1], SA.shape[2]
    n = SB.shape[1]
    assert k * s * 127 * 127 < 2**53
    A64 = SA.astype(np.float64)
    B64 = SB.astype(np.float64)
    out = np.zeros((t - 1, m, n), dtype=np.int64)
    for L in range(2, t + 1):
        acc = np.zeros((m, n), dtype=np.float64)
        for p in range(1, sa + 1):
            q = L - p
            if 1 <= q <= sb:
                acc += A64[p - 1] @ B64[q - 1].T
        out[L - 2] = acc.astype(np.int64)
    return out


def combine_levels(I, t):
    """Exact T = sum_{L=2..t} I_L * 2**(7(t-L)) as a numpy object array of Python ints."""
    T = np.zeros(I.shape[1:], dtype=object)
    for L in range(2, t + 1):
        T = T + I[L - 2].astype(object) * (1 << (BITS * (t - L)))
    return T


def _rn_scaled(T, sh):
    """Correctly rounded float of the exact rational T * 2**sh (Python int T)."""
    if T == 0:
        return 0.0
    try:
        if sh >= 0:
            return float(T << sh)
        return T / (1 << (-sh))
    except OverflowError:
        return math.copysign(math.inf, T)


def rounded_products(I, e, f, s, t=None):
    """D = RN(T * 2**(e_i + f_j - 7t)) as float64 [m, n] (NaN for NONFINITE scales)."""
    t = s + 1 if t is None else t
    T = combine_levels(I, t)
    m, n = T.shape
    e = np.asarray(e, dtype=np.int64)
    f = np.asarray(f, dtype=np.int64)
    D = np.empty((m, n), dtype=np.float64)
    for i in range(m):
        for j in range(n):
            if e[i] == NONFINITE or f[j] == NONFINITE:
                D[i, j] = np.nan
            else:
                D[i, j] = _rn_scaled(int(T[i, j]), int(e[i]) + int(f[j]) - BITS * t)
    return D


def recombine(I, e, f, s, t=None, alpha=1.0, beta=0.0, C=None):
    """out = RN(RN(alpha*D) + RN(beta*C)) with D from rounded_products."""
    D = rounded_products(I, e, f, s, t)
    with np.errstate(all="ignore"):
        ad = np.float64(alpha) * D
        if beta == 0.0:
            return ad
        return ad + np.float64(beta) * np.asarray(C, dtype=np.float64)


def emul_gemm(A, B, s, alpha=1.0, beta=0.0, C=None, t=None):
    """beta*C + alpha*(A @ B) emulated with s INT8 slices per operand (A: m x k, B: k x n)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    t = s + 1 if t is None else t
    e, SA = split_rows(A, s)
    f, SB = split_cols(B, s)
    I = level_sums(SA, SB, t)
    if beta != 0.0:
        C = np.asarray(C, dtype=np.float64)
    return recombine(I, e, f, s, t=t, alpha=alpha, beta=beta, C=C)


def emul_gemm_unequal(A, B, sa, sb, alpha=1.0, beta=0.0, C=None, t=None):
    """beta*C + alpha*(A @ B) with sa slices of A and sb slices of B.

    Reading of the unequal split counts the paper cites among the accuracy
    extensions (Section 3): both operands are split with s = max(sa, sb)
    slices, whose leading sa (sb) slices are exactly the slices of an sa-slice
    (sb-slice) split, and only the pairs with p <= sa, q <= sb and p + q <= t
    are kept (t defaults to s + 1).  With t = sa + sb every such pair is kept
    and the kept sum is the exact product of the sa-digit and sb-digit scaled
    integers.  Recombination and C update as in emul_gemm.
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    s = max(sa, sb)
    t = s + 1 if t is None else t
    e, SA = split_rows(A, s)
    f, SB = split_cols(B, s)
    I = level_sums(SA, SB, t, sa=sa, sb=sb)
    if beta != 0.0:
        C = np.asarray(C, dtype=np.float64)
    return recombine(I, e, f, s, t=t, alpha=alpha, beta=beta, C=C)


def emul_product_exact(A, B, s, t=None):
    """The exact (unrounded) kept-level product as Fractions, for pins."""
    from fractions import Fraction
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    t = s + 1 if t is None else t
    e, SA = split_rows(A, s)
    f, SB = split_cols(B, s)
    T = combine_levels(level_sums(SA, SB, t), t)
    m, n = T.shape
    return [[Fraction(int(T[i, j])) * Fraction(2) ** (int(e[i]) + int(f[j]) - BITS * t)
             for j in range(n)] for i in range(m)]
