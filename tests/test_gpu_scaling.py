"""Eq. 4 of arXiv 2509.23565 through the GPU product: (L_A A R_A)(L_B B R_B)
with diagonal or permutation matrices, at sizes that span several tiles and
ragged tails.  Outer power-of-two scalings and permutations (rows of A,
columns of B, k jointly) must leave the emulated product exactly unchanged up
to the same scaling / permutation of the result; an inner scaling along k must
give the oracle's result bit for bit and lose accuracy against the exact
product as its range grows.
"""
import numpy as np
import pytest

from oracle import emulgemm, exact
from paper_2509_23565_gb300 import inputs
from paper_2509_23565_gb300.binding import ColMajor

pytestmark = pytest.mark.gpu


def _gemm(gpu_lib, A, B, s):
    dC = ColMajor.from_numpy(np.zeros((A.shape[0], B.shape[1]), order="F"))
    gpu_lib.dgemm(ColMajor.from_numpy(np.asfortranarray(A)), ColMajor.from_numpy(np.asfortranarray(B)), dC, s)
    gpu_lib.sync_status()
    return dC.numpy()


def _same_bits(a, b):
    return np.array_equal(np.asarray(a, dtype=np.float64).view(np.int64), np.asarray(b, dtype=np.float64).view(np.int64))


@pytest.mark.parametrize("s", [4, 7])
def test_outer_scaling_and_permutations_exact(gpu_lib, s):
    m, k, n = 300, 257, 200
    A, B = inputs.uniform(m, k, seed=431), inputs.uniform(k, n, seed=432)
    rng = np.random.default_rng(433)
    D0 = _gemm(gpu_lib, A, B, s)
    a, b = rng.integers(-40, 41, size=m), rng.integers(-40, 41, size=n)
    D1 = _gemm(gpu_lib, np.ldexp(A, a[:, None]), np.ldexp(B, b[None, :]), s)
    assert _same_bits(D1, np.ldexp(np.ldexp(D0, a[:, None]), b[None, :]))
    p, q, r = rng.permutation(m), rng.permutation(k), rng.permutation(n)
    D2 = _gemm(gpu_lib, A[p][:, q], B[q][:, r], s)
    assert _same_bits(D2, D0[p][:, r])


def test_inner_scaling_matches_oracle_and_degrades(gpu_lib):
    m, k, n, s = 160, 96, 140, 6
    A, B = inputs.uniform(m, k, seed=441), inputs.uniform(k, n, seed=442)
    rng = np.random.default_rng(443)
    rows, cols = rng.choice(m, 12, replace=False), rng.choice(n, 12, replace=False)
    absprod = exact.abs_product(A, B)
    errs = []
    for r in (0, 8, 16):
        d = rng.integers(-r, r + 1, size=k)
        As, Bs = np.ldexp(A, d[None, :]), np.ldexp(B, -d[:, None])
        D = _gemm(gpu_lib, As, Bs, s)
        assert _same_bits(D, emulgemm.emul_gemm(As, Bs, s))
        err = max(abs(float(D[i, j]) - float(exact.exact_entry(A, B, i, j))) / absprod[i, j]
                  for i in rows for j in cols)
        errs.append(err)
    assert errs[0] < errs[1] < errs[2] and errs[2] > 2.0 ** 10 * errs[0], errs
