"""Scale extraction and slicing: Section 2 of arXiv 2509.23565 (Eq. 1-4).

The paper splits the 53-bit FP64 significand of every entry into several
8-bit integer pieces (Eq. 1 for two pieces, Eq. 2 for k pieces) and notes that
fixed-width pieces carry no exponent, so each row of A / column of B needs its
own power-of-two scale (the range example of Eq. 3 and the scaling of Eq. 4).
The paper leaves the exact split unspecified; this oracle takes the reading:

* scale: e_i = the smallest integer e with max_j |a_ij| < 2**e  (all-zero row:
  e_i = 0; a row holding Inf or NaN: e_i = NONFINITE);
* W = 7*s bits; N_ij = trunc(a_ij * 2**(W - e_i)) (toward zero), |N_ij| < 2**W;
* slice p = 1..s (p = 1 most significant):
  S_p = sign(a_ij) * ((|N_ij| >> 7*(s-p)) & 127), an INT8 value in [-127, 127].

Test infrastructure only (see the package docstring).
"""
import numpy as np

BITS = 7                 # magnitude bits per INT8 slice; the sign rides along
NONFINITE = 2**31 - 1    # scale sentinel for a row / column holding Inf or NaN


def row_exponents(A):
    """e_i = smallest integer e with max_j |a_ij| < 2**e, per row of A (m x k).

    np.frexp(x) returns (f, ex) with x = f * 2**ex and 0.5 <= |f| < 1, hence
    x < 2**ex and x >= 2**(ex-1): ex is exactly the smallest such e, also for
    subnormal x.
    """
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    e = np.zeros(m, dtype=np.int64)
    if A.shape[1] == 0 or m == 0:
        return e
    finite = np.isfinite(A).all(axis=1)
    mx = np.where(finite, np.abs(np.where(np.isfinite(A), A, 0.0)).max(axis=1), 0.0)
    _, ex = np.frexp(mx)
    e[:] = ex
    e[mx == 0.0] = 0
    e[~finite] = NONFINITE
    return e


def col_exponents(B):
    """f_j = smallest integer f with max_k |b_kj| < 2**f, per column of B (k x n)."""
    return row_exponents(np.asarray(B, dtype=np.float64).T)


def scaled_integers(A, e, s):
    """N_ij = trunc(a_ij * 2**(7s - e_i)) computed exactly in int64.

    a = M * 2**(ex - 53) with M = f * 2**53 an integer (|M| < 2**53), so
    N = trunc(M * 2**sh) with sh = ex - 53 + W - e_i; since |a| < 2**e_i,
    sh <= W - 53 <= 3 for s <= 8, so the left shift never overflows.
    Rows with e_i == NONFINITE give N = 0 (their products are NaN anyway).
    """
    A = np.asarray(A, dtype=np.float64)
    W = BITS * s
    e = np.asarray(e, dtype=np.int64)
    bad = e == NONFINITE
    Af = np.where(np.isfinite(A), A, 0.0)
    Af[bad, :] = 0.0
    f, ex = np.frexp(Af)
    M = (f * 2.0**53).astype(np.int64)
    sh = ex.astype(np.int64) - 53 + W - np.where(bad, 0, e)[:, None]
    mag = np.abs(M)
    left = np.clip(sh, 0, 62)
    right = np.clip(-sh, 0, 63)
    mag = np.where(sh >= 0, mag << left, mag >> right)
    return np.where(M < 0, -mag, mag)


def digits(N, s):
    """Signed 7-bit digits of N: S[p-1] = sign(N) * ((|N| >> 7(s-p)) & 127)."""
    N = np.asarray(N, dtype=np.int64)
    mag = np.abs(N)
    sgn = np.where(N < 0, -1, 1)
    out = np.empty((s,) + N.shape, dtype=np.int8)
    for p in range(1, s + 1):
        out[p - 1] = (sgn * ((mag >> (BITS * (s - p))) & 127)).astype(np.int8)
    return out


def split_rows(A, s):
    """Slices of A by rows: (e[m], S[s, m, k]) with a_ik ~ 2**e_i * sum_p S_p 2**(-7p)."""
    e = row_exponents(A)
    return e, digits(scaled_integers(A, e, s), s)


def split_cols(B, s):
    """Slices of B by columns: (f[n], S[s, n, k]); S[:, j, :] holds column j of B."""
    B = np.asarray(B, dtype=np.float64)
    f = col_exponents(B)
    return f, digits(scaled_integers(B.T, f, s), s)


def reconstruct(S, e):
    """Exact value sum_p S_p 2**(e - 7p) as a list of Python Fractions (pins only)."""
    from fractions import Fraction
    s = S.shape[0]
    rows = S.shape[1]
    out = []
    for i in range(rows):
        row = []
        for k in range(S.shape[2]):
            acc = 0
            for p in range(1, s + 1):
                acc = acc * 128 + int(S[p - 1, i, k])
            row.append(Fraction(acc) * Fraction(2) ** (int(e[i]) - BITS * s))
        out.append(row)
    return out
