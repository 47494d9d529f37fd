"""Factorizations at the sizes the benchmark runs, checked by the oracle's residuals.

The headline configuration factors n = 16384 and 32768 matrices; the oracle
cannot redo those factorizations, so what is checked is what the paper's
Section 4 asks of them and what the oracle can compute one row at a time:

* the backward error ||Ax - b|| / (||A|| ||x|| n eps) and the scaled residual
  of Eq. 8 of the solve, both computed on the CPU from A, x and b;
* the factorization residual ||PA - LU|| (LU) or ||A - LL^T|| (Cholesky) over
  ||A|| n eps, on sampled rows (first, last and random rows);
* the device residual kernel against the oracle's formula at this size;
* info = 0 and a valid pivot vector.

Inputs follow the configurations of the method's sweeps: U(-1, 1), the
log-scaled generator u 10^e with e ~ U(-16, 16), and SPD matrices
Q diag(lam) Q^T with condition number 1e12, all drawn on the GPU with seeded
torch generators (drawing 2 GB on the host takes minutes).
"""
import numpy as np
import pytest

from oracle import residual
from paper_2509_23565_gb300 import inputs
from paper_2509_23565_gb300.binding import ColMajor

pytestmark = pytest.mark.gpu

N = 16384


def _rows(n, seed, count=30):
    rng = np.random.default_rng(seed)
    return np.sort(np.concatenate([[0, n - 1], rng.choice(np.arange(1, n - 1), count, replace=False)]))


def _lu_check(gpu_lib, store, b, nb, s, factor_bound):
    """store: the column-major device store of A (row j = column j)."""
    n = store.shape[0]
    A = store.cpu().numpy().T            # the matrix itself, on the host
    dA = ColMajor(store.clone(), n, n)
    ipiv, info = gpu_lib.dgetrf(dA, nb=nb, slices=s)
    db = ColMajor.from_numpy(b)
    gpu_lib.dgetrs(dA, ipiv, db)
    dev = gpu_lib.backward_error(ColMajor(store, n, n), db, ColMajor.from_numpy(b)).cpu().numpy()
    gpu_lib.sync_status()
    assert int(info.item()) == 0
    piv = ipiv.cpu().numpy()
    assert (piv >= np.arange(1, n + 1)).all() and (piv <= n).all()
    x = db.numpy()[:, 0]
    berr = residual.backward_error(A, x, b)
    eq8 = residual.scaled_residual(A, x, b)
    assert berr < 16 and eq8 < 16, (berr, eq8)
    assert abs(dev[0] - eq8) <= 1e-9 * max(1.0, eq8) and abs(dev[1] - berr) <= 1e-9 * max(1.0, berr)
    LU = dA.numpy()
    del dA
    fres = residual.lu_residual_rows(A, LU, piv, _rows(n, 7))
    assert fres < factor_bound, fres
    return berr, fres


def test_lu_16384_uniform_s7(gpu_lib):
    """The headline generator: U(-1, 1), nb = 256, s = 7."""
    b = inputs.vector(N, seed=16002)
    _lu_check(gpu_lib, inputs.uniform_device(N, N, seed=16001), b, 256, 7, 100)


def test_lu_16384_uniform_nb512_s7(gpu_lib):
    """nb = 512: 512-column panels factored as two halves, trailing updates
    with k = 512."""
    b = inputs.vector(N, seed=16004)
    _lu_check(gpu_lib, inputs.uniform_device(N, N, seed=16003), b, 512, 7, 100)


def test_lu_16384_log_scaled_r16_s7(gpu_lib):
    """u 10^e, e ~ U(-16, 16): entries spread over about 106 binades.  Per-row
    and per-column scales keep every update normwise accurate (entries far
    below their row's largest lose their low bits, but they are also far
    below ||A||), so the backward error stays under 16 at 7 slices."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(16011)
    b = inputs.vector(N, seed=16012)
    _lu_check(gpu_lib, inputs.log_scaled_device(N, N, 16, gen), b, 256, 7, 100)


def test_cholesky_16384_cond1e12_s7(gpu_lib):
    """SPD A = Q diag(lam) Q^T, lam log-spaced from 1 to 1e-12 (formed on the
    GPU in FP64 by torch), lower Cholesky with nb = 256 and s = 7."""
    import torch
    n = N
    dA0 = inputs.spd_device(n, 1e12, seed=16021)
    A = dA0.cpu().numpy()                # symmetric: the store is the matrix
    b = inputs.vector(n, seed=16022)
    dA = ColMajor(dA0.clone(), n, n)
    info = gpu_lib.dpotrf(dA, nb=256, slices=7)
    db = ColMajor.from_numpy(b)
    gpu_lib.dpotrs(dA, db)
    dev = gpu_lib.backward_error(ColMajor(dA0, n, n), db, ColMajor.from_numpy(b)).cpu().numpy()
    gpu_lib.sync_status()
    assert int(info.item()) == 0
    x = db.numpy()[:, 0]
    berr = residual.backward_error(A, x, b)
    eq8 = residual.scaled_residual(A, x, b)
    assert berr < 16 and eq8 < 16, (berr, eq8)
    # x is of order 1e12 here, so A x - b cancels to about 1e-12 of |A||x|: the
    # device kernel and numpy sum the products of A x in different orders and
    # agree only to the rounding of A x, which in these units (||A|| ||x|| n eps)
    # is about 1 / sqrt(n) for random rounding errors
    assert abs(dev[1] - berr) <= 1e-2, (dev[1], berr)
    L = dA.numpy()
    # the strictly upper triangle is not touched
    assert np.array_equal(np.triu(L, 1), np.triu(A, 1))
    del dA, dA0
    torch.cuda.empty_cache()
    fres = residual.chol_residual_rows(A, L, _rows(n, 8))
    assert fres < 16, fres
