"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

Holds no arithmetic of the emulation method: only random draws and the matrix
families of arXiv 2509.23565.  Every generator returns float64 numpy arrays in
column-major (Fortran) order, the layout of the C-ABI.

* uniform(m, n, seed, lo, hi)      iid U(lo, hi) entries (HPL draws U(-1/2, 1/2),
                                   Section 6; the dynamic-range sweeps use U(-1, 1)).
* log_scaled(m, n, r, seed)        u * 10**e, u ~ U(-1, 1), e ~ U(-r, r) continuous.
* spd(n, cond, seed)               Q diag(lam) Q^T, Q from the QR of a Gaussian
                                   matrix, lam log-spaced from 1 to 1/cond.
* wilkinson(n)                     Eq. 9 (diagonal 1, -1 below, 1 in the last column).
* turing(n)                        the matrix of Eq. 10 (no last-column 1's).
* parawilk(n, d, b, alpha)         Section 5: d subdiagonals of -1, alpha above the
                                   diagonal in every b-th column (1-based j = 1+b, 1+2b, ...)
                                   and in the last column (Eq. 11, 13).
* parawilk_random(n, d, b, alpha, seed)
                                   Eq. 15: 2 u**2 (u ~ U(0, 1)) in the zero
                                   positions of parawilk, parawilk elsewhere.
* uniform_device, log_scaled_device
                                   the same distributions drawn on the GPU with a seeded
                                   torch.Generator (column-major device stores).
* spd_device(n, cond, seed)        the spd() recipe drawn and formed on the GPU in FP64
                                   (torch: seeded normal draws, QR, Q diag(lam) Q^T) for the
                                   large sizes; returned as a device tensor (symmetric, so
                                   row-major and column-major storage coincide).
* diag_dominant(n, seed)           U(-1, 1) entries with n on the diagonal: strictly
                                   diagonally dominant by rows and columns, so
                                   elimination needs no pivoting (the no-pivot LU).
* bidiag_factors(n, seed, zero_at) unit lower bidiagonal L and upper bidiagonal U
                                   with integer entries (subdiagonal / superdiagonal
                                   in {-1, 0, 1}, diagonal of U +-1, or 0 at zero_at)
                                   and A = L U: every Schur complement and block
                                   inverse of A is a small integer matrix.
"""
import numpy as np


def _rng(seed):
    return np.random.default_rng(seed)


def uniform(m, n, seed, lo=-1.0, hi=1.0):
    rng = _rng(seed)
    x = rng.random((n, m))                        # generated column by column
    x *= (hi - lo)
    x += lo
    return np.asfortranarray(x.T)


def log_scaled(m, n, r, seed):
    rng = _rng(seed)
    u = rng.random((n, m)) * 2.0 - 1.0
    u[u == 0.0] = 0.5
    e = (rng.random((n, m)) * 2.0 - 1.0) * r
    return np.asfortranarray((u * np.power(10.0, e)).T)


def vector(n, seed, lo=-1.0, hi=1.0):
    rng = _rng(seed)
    return rng.random(n) * (hi - lo) + lo


def spd(n, cond, seed):
    rng = _rng(seed)
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]
    lam = np.logspace(0.0, -np.log10(cond), n)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A)


def spd_device(n, cond, seed, device="cuda"):
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    G = torch.randn((n, n), generator=gen, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    del G
    Q *= torch.sign(torch.diagonal(R))[None, :]
    del R
    lam = torch.logspace(0.0, -float(np.log10(cond)), n, device=device, dtype=torch.float64)
    A = (Q * lam[None, :]) @ Q.T
    del Q
    A = 0.5 * (A + A.T)
    return A.contiguous()


def turing(n):
    A = np.eye(n) - np.tril(np.ones((n, n)), -1)
    return np.asfortranarray(A)


def wilkinson(n):
    A = turing(n)
    A[:, n - 1] = 1.0
    return np.asfortranarray(A)


def parawilk(n, d, b, alpha):
    A = np.eye(n)
    for k in range(1, min(d, n - 1) + 1):
        A -= np.eye(n, k=-k)
    cols = [j for j in range(1, n) if j % b == 0] + [n - 1]   # 0-based: 1-based j = 1+b, 1+2b, ..., n
    for j in set(cols):
        A[:j, j] = alpha
    return np.asfortranarray(A)


def parawilk_random(n, d, b, alpha, seed):
    P = parawilk(n, d, b, alpha)
    rng = _rng(seed)
    u = rng.random((n, n)).T
    fill = 2.0 * u * u
    return np.asfortranarray(np.where(P == 0.0, fill, P))


def batch_sizes(count, lo, hi, seed):
    """Log-uniform integer sizes in [lo, hi] for the batched solver."""
    rng = _rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), count))).astype(np.int64).clip(lo, hi)


def uniform_device(m, n, seed, lo=-1.0, hi=1.0, device="cuda"):
    """iid U(lo, hi) drawn on the device with a seeded torch.Generator;
    returned as a column-major store (n x m tensor: row j is column j).  For
    the large sizes, where drawing on the host takes minutes."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    x = torch.rand((n, m), generator=gen, device=device, dtype=torch.float64)
    x *= (hi - lo)
    x += lo
    return x


def log_scaled_device(m, n, r, gen, device="cuda"):
    """u * 10**e (u ~ U(-1, 1), e ~ U(-r, r)) drawn on the device with a seeded
    torch.Generator; returned as a column-major store (n x m tensor: row j is
    column j).  Used for bulk training data of the slice selector."""
    import torch
    u = torch.rand((n, m), generator=gen, device=device, dtype=torch.float64) * 2.0 - 1.0
    if r == 0:
        return u
    e = (torch.rand((n, m), generator=gen, device=device, dtype=torch.float64) * 2.0 - 1.0) * r
    return u * torch.pow(10.0, e)


def mixed_range(n, nb, ranges, seed):
    """Uniform(-1, 1) matrix whose block rows (nb rows each) are scaled
    entrywise by 10**e, e ~ U(-r, r), with r drawn per block row from `ranges`
    (mixed blocks, e.g. r in {0, 8, 16})."""
    rng = _rng(seed)
    A = rng.random((n, n)) * 2.0 - 1.0
    for i0 in range(0, n, nb):
        r = ranges[rng.integers(len(ranges))]
        if r:
            rows = slice(i0, min(n, i0 + nb))
            A[rows, :] *= np.power(10.0, (rng.random((A[rows, :].shape)) * 2.0 - 1.0) * r)
    return np.asfortranarray(A)


def diag_dominant(n, seed):
    A = uniform(n, n, seed)
    A[np.arange(n), np.arange(n)] = float(n)
    return A


def bidiag_factors(n, seed, zero_at=None):
    rng = _rng(seed)
    L = np.eye(n)
    U = np.diag(rng.choice([-1.0, 1.0], size=n))
    if n > 1:
        L[np.arange(1, n), np.arange(n - 1)] = rng.integers(-1, 2, size=n - 1).astype(np.float64)
        U[np.arange(n - 1), np.arange(1, n)] = rng.integers(-1, 2, size=n - 1).astype(np.float64)
    if zero_at is not None:
        U[zero_at, zero_at] = 0.0
    return np.asfortranarray(L), np.asfortranarray(U), np.asfortranarray(L @ U)
