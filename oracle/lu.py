"""Blocked factorizations and solves (Section 4, Eq. 5-7 of arXiv 2509.23565).

The paper factors A with the 2-by-2 partition of Eq. 6; after the panel
[A11; A21] is factored with partial pivoting (L11 unit lower with entries of
magnitude at most 1, U11 upper) and U12 = L11^{-1} A12, all third-order work is
the Schur complement of Eq. 7, A22 <- A22 - L21 U12, which is the part the
split-integer product replaces.  The paper also names symmetric positive
definite matrices as a case the method applies to; ``potrf`` is blocked
Cholesky with the same structure (A22 <- A22 - L21 L21^T).

``update`` selects how the trailing update is computed:
  "fp64"      plain FP64 (numpy matmul);
  "emulated"  the split-integer product of ``emulgemm`` with s slices.
Pivot choice: the first index of the largest |a| in the column (LAPACK idamax).
A zero pivot leaves the column unscaled and sets info to its 1-based index
(the first one), as LAPACK dgetrf does.

Test infrastructure only (see the package docstring).
"""
import numpy as np
from scipy.linalg import solve_triangular

from . import emulgemm


def _trailing_update(L21, U12, A22, update, s):
    if update == "fp64":
        return A22 - L21 @ U12
    if update == "emulated":
        return emulgemm.emul_gemm(L21, U12, s, alpha=-1.0, beta=1.0, C=A22)
    raise ValueError(update)


def getf2(P, ipiv_out, info_state, offset):
    """Unblocked partial-pivot LU of the panel P (m x b), in place.

    ipiv_out[j] receives the 1-based row index (within P, shifted by offset)
    of the pivot of column j; info_state[0] receives the first zero pivot.
    """
    m, b = P.shape
    for j in range(min(m, b)):
        col = np.abs(P[j:, j])
        p = j + int(np.argmax(col))            # first maximal index
        ipiv_out[j] = offset + p + 1
        if P[p, j] != 0.0:
            if p != j:
                P[[j, p], :] = P[[p, j], :]
            P[j + 1:, j] = P[j + 1:, j] / P[j, j]
        elif info_state[0] == 0:
            info_state[0] = offset + j + 1
        if j + 1 < b:
            P[j + 1:, j + 1:] -= np.outer(P[j + 1:, j], P[j, j + 1:])


def getrf(A, nb=64, update="fp64", s=7):
    """Right-looking blocked LU with partial pivoting.  Returns (LU, ipiv, info)."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    assert A.shape == (n, n)
    ipiv = np.zeros(n, dtype=np.int64)
    info = [0]
    for j0 in range(0, n, nb):
        jb = min(nb, n - j0)
        panel = A[j0:, j0:j0 + jb]
        piv = np.zeros(jb, dtype=np.int64)
        getf2(panel, piv, info, j0)
        ipiv[j0:j0 + jb] = piv
        # apply the panel's row interchanges to the columns left and right of it
        for j in range(j0, j0 + jb):
            p = ipiv[j] - 1
            if p != j:
                A[[j, p], :j0] = A[[p, j], :j0]
                A[[j, p], j0 + jb:] = A[[p, j], j0 + jb:]
        if j0 + jb < n:
            L11 = A[j0:j0 + jb, j0:j0 + jb]
            A[j0:j0 + jb, j0 + jb:] = solve_triangular(L11, A[j0:j0 + jb, j0 + jb:],
                                                       lower=True, unit_diagonal=True)
            L21 = A[j0 + jb:, j0:j0 + jb]
            U12 = A[j0:j0 + jb, j0 + jb:]
            A[j0 + jb:, j0 + jb:] = _trailing_update(L21, U12, A[j0 + jb:, j0 + jb:], update, s)
    return A, ipiv, info[0]


def getf2_nopiv(P, info_state, offset):
    """Unblocked LU without pivoting of the panel P (m x b), in place; a zero
    pivot leaves its column unscaled and sets info_state[0] (the first one)."""
    m, b = P.shape
    for j in range(min(m, b)):
        if P[j, j] != 0.0:
            P[j + 1:, j] = P[j + 1:, j] / P[j, j]
        elif info_state[0] == 0:
            info_state[0] = offset + j + 1
        if j + 1 < b:
            P[j + 1:, j + 1:] -= np.outer(P[j + 1:, j], P[j, j + 1:])


def getrf_nopiv(A, nb=64, update="fp64", s=7):
    """Right-looking blocked LU without pivoting, the Level-3-only variant of
    Section 8: panel by unblocked elimination, U12 = L11^{-1} A12, then the
    Schur complement of Eq. 7.  Returns (LU, info)."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    assert A.shape == (n, n)
    info = [0]
    for j0 in range(0, n, nb):
        jb = min(nb, n - j0)
        getf2_nopiv(A[j0:, j0:j0 + jb], info, j0)
        if j0 + jb < n:
            L11 = A[j0:j0 + jb, j0:j0 + jb]
            A[j0:j0 + jb, j0 + jb:] = solve_triangular(L11, A[j0:j0 + jb, j0 + jb:],
                                                       lower=True, unit_diagonal=True)
            L21 = A[j0 + jb:, j0:j0 + jb]
            U12 = A[j0:j0 + jb, j0 + jb:]
            A[j0 + jb:, j0 + jb:] = _trailing_update(L21, U12, A[j0 + jb:, j0 + jb:], update, s)
    return A, info[0]


def getrs(LU, ipiv, b):
    """Solve A x = b from getrf's output (row interchanges, then L, then U)."""
    LU = np.asarray(LU, dtype=np.float64)
    x = np.array(b, dtype=np.float64, copy=True)
    for j, p in enumerate(np.asarray(ipiv) - 1):
        if p != j:
            x[[j, p]] = x[[p, j]]
    x = solve_triangular(LU, x, lower=True, unit_diagonal=True)
    return solve_triangular(LU, x, lower=False)


def potf2(D, info_state, offset):
    """Unblocked lower Cholesky of the diagonal block D (b x b), in place."""
    b = D.shape[0]
    for j in range(b):
        d = D[j, j] - np.dot(D[j, :j], D[j, :j])
        if not d > 0.0:
            D[j, j] = d
            if info_state[0] == 0:
                info_state[0] = offset + j + 1
            return False
        D[j, j] = np.sqrt(d)
        if j + 1 < b:
            D[j + 1:, j] = (D[j + 1:, j] - D[j + 1:, :j] @ D[j, :j]) / D[j, j]
    return True


def potrf(A, nb=64, update="fp64", s=7):
    """Right-looking blocked lower Cholesky.  Returns (L, info); only the lower
    triangle of the result is meaningful."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    info = [0]
    for j0 in range(0, n, nb):
        jb = min(nb, n - j0)
        if not potf2(A[j0:j0 + jb, j0:j0 + jb], info, j0):
            break
        if j0 + jb < n:
            L11 = A[j0:j0 + jb, j0:j0 + jb]
            # L21 = A21 L11^{-T}
            A[j0 + jb:, j0:j0 + jb] = solve_triangular(L11, A[j0 + jb:, j0:j0 + jb].T, lower=True).T
            L21 = A[j0 + jb:, j0:j0 + jb]
            A[j0 + jb:, j0 + jb:] = _trailing_update(L21, L21.T, A[j0 + jb:, j0 + jb:], update, s)
    return np.tril(A), info[0]


def potrs(L, b):
    """Solve A x = b from the lower Cholesky factor."""
    L = np.tril(np.asarray(L, dtype=np.float64))
    y = solve_triangular(L, np.asarray(b, dtype=np.float64), lower=True)
    return solve_triangular(L.T, y, lower=False)
