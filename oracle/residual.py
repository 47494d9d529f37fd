"""Residual measures for the solve of Eq. 5 (Section 4, Eq. 8 of arXiv 2509.23565).

* scaled_residual: Eq. 8, ||Ax-b||_inf / ((||A||_inf ||x||_inf + ||b||_inf) n eps),
  which the paper requires to be below 16 for a valid HPL run.
* backward_error: ||Ax-b||_inf / (||A||_inf ||x||_inf n eps) (same without the
  ||b|| term, hence never smaller than Eq. 8).
* lu_residual / chol_residual: factorization residuals ||PA - LU||_inf /
  (||A||_inf n eps) and ||A - LL^T||_inf / (||A||_inf n eps).
* lu_residual_rows / chol_residual_rows: the same quotient with the infinity
  norm of the numerator taken over the given rows only (a lower bound of the
  full residual, for sizes where the full product L U is too costly here).

Reading: eps = 2**-53, the unit roundoff of FP64 (LAPACK dlamch('E')), which the
paper does not define.

Test infrastructure only (see the package docstring).
"""
import numpy as np

EPS = 2.0 ** -53


def _inf_norm(M):
    M = np.asarray(M, dtype=np.float64)
    if M.ndim == 1:
        return float(np.max(np.abs(M))) if M.size else 0.0
    return float(np.max(np.sum(np.abs(M), axis=1))) if M.size else 0.0


def residual_vector(A, x, b):
    return np.asarray(A, dtype=np.float64) @ np.asarray(x, dtype=np.float64) - np.asarray(b, dtype=np.float64)


def scaled_residual(A, x, b):
    """Eq. 8."""
    n = np.asarray(A).shape[0]
    r = residual_vector(A, x, b)
    den = (_inf_norm(A) * _inf_norm(x) + _inf_norm(b)) * n * EPS
    return _inf_norm(r) / den


def backward_error(A, x, b):
    """||Ax-b|| / (||A|| ||x|| n eps)."""
    n = np.asarray(A).shape[0]
    r = residual_vector(A, x, b)
    den = _inf_norm(A) * _inf_norm(x) * n * EPS
    return _inf_norm(r) / den


def unpack_lu(LU):
    LU = np.asarray(LU, dtype=np.float64)
    L = np.tril(LU, -1) + np.eye(LU.shape[0])
    U = np.triu(LU)
    return L, U


def permutation_from_ipiv(ipiv, n):
    """Row order perm such that (P A) = A[perm] for LAPACK-style 1-based ipiv."""
    perm = np.arange(n)
    for j, p in enumerate(np.asarray(ipiv) - 1):
        perm[[j, p]] = perm[[p, j]]
    return perm


def lu_residual(A, LU, ipiv):
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    L, U = unpack_lu(LU)
    PA = A[permutation_from_ipiv(ipiv, n)]
    return _inf_norm(PA - L @ U) / (_inf_norm(A) * n * EPS)


def chol_residual(A, Lfac):
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    L = np.tril(np.asarray(Lfac, dtype=np.float64))
    return _inf_norm(A - L @ L.T) / (_inf_norm(A) * n * EPS)


def lu_residual_rows(A, LU, ipiv, rows):
    """max over the given rows i of sum_j |(PA - LU)_ij|, over ||A||_inf n eps."""
    A = np.asarray(A, dtype=np.float64)
    LU = np.asarray(LU, dtype=np.float64)
    n = A.shape[0]
    rows = np.asarray(rows)
    perm = permutation_from_ipiv(ipiv, n)
    cols = np.arange(n)[None, :]
    Lr = np.where(cols < rows[:, None], LU[rows, :], 0.0)     # strictly lower part of row i of L
    Lr[np.arange(len(rows)), rows] = 1.0                        # unit diagonal
    R = A[perm[rows], :] - Lr @ np.triu(LU)
    return float(np.max(np.sum(np.abs(R), axis=1))) / (_inf_norm(A) * n * EPS)


def chol_residual_rows(A, Lfac, rows):
    """max over the given rows i of sum_j |(A - LL^T)_ij|, over ||A||_inf n eps."""
    A = np.asarray(A, dtype=np.float64)
    L = np.tril(np.asarray(Lfac, dtype=np.float64))
    n = A.shape[0]
    rows = np.asarray(rows)
    R = A[rows, :] - L[rows, :] @ L.T
    return float(np.max(np.sum(np.abs(R), axis=1))) / (_inf_norm(A) * n * EPS)
