"""Eq. 4 of arXiv 2509.23565 (Sec. 2): both product operands scaled,
(L_A A R_A)(L_B B R_B), by diagonal or permutation matrices, which FP64 takes
in its stride.  With one power-of-two scale per row of A and per column of B
(the reading of the split), the oracle's emulated product must show:

* outer power-of-two scalings L_A, R_B pass through exactly;
* permutations of the rows of A, of the columns of B, and of k (jointly in A
  and B) pass through exactly: the level sums are exact integers;
* the inner scaling R_A L_B (a diagonal along k) widens the range inside the
  rows of A and the columns of B; the error against the exact product grows
  with that range and stays within the a-priori bound.
"""
import numpy as np
import pytest

from oracle import bounds, emulgemm, exact
from paper_2509_23565_gb300 import inputs


def _pair(m, k, n, seed):
    return inputs.uniform(m, k, seed=seed), inputs.uniform(k, n, seed=seed + 1)


@pytest.mark.parametrize("s", [3, 5, 7])
def test_outer_power_of_two_scaling_exact(s):
    A, B = _pair(40, 70, 30, seed=401)
    rng = np.random.default_rng(402)
    a = rng.integers(-30, 31, size=40)
    b = rng.integers(-30, 31, size=30)
    D0 = emulgemm.emul_gemm(A, B, s)
    D1 = emulgemm.emul_gemm(np.ldexp(A, a[:, None]), np.ldexp(B, b[None, :]), s)
    assert np.array_equal(D1, np.ldexp(np.ldexp(D0, a[:, None]), b[None, :]))


@pytest.mark.parametrize("s", [3, 7])
def test_permutations_exact(s):
    A, B = _pair(33, 65, 29, seed=411)
    rng = np.random.default_rng(412)
    p, q, r = rng.permutation(33), rng.permutation(65), rng.permutation(29)
    D0 = emulgemm.emul_gemm(A, B, s)
    D1 = emulgemm.emul_gemm(A[p][:, q], B[q][:, r], s)
    assert np.array_equal(D1, D0[p][:, r])


def test_inner_scaling_degrades_within_bound():
    """d_k uniform in [-r, r]: (A 2^d)(2^-d B) = AB exactly, but each row of
    A 2^d now spans about 2r binades, and the entries far below the row's
    scale lose their low bits in the split."""
    m, k, n, s = 16, 48, 16, 6
    A, B = _pair(m, k, n, seed=421)
    AB = exact.exact_product(A, B)
    absprod = exact.abs_product(A, B)
    rng = np.random.default_rng(422)
    errs = []
    for r in (0, 6, 12, 18):
        d = rng.integers(-r, r + 1, size=k)
        As, Bs = np.ldexp(A, d[None, :]), np.ldexp(B, -d[:, None])
        D = emulgemm.emul_gemm(As, Bs, s)
        err = np.array([[abs(float(D[i, j]) - float(AB[i][j])) for j in range(n)] for i in range(m)])
        assert np.all(err <= bounds.emul_bound(As, Bs, s, D) * (1 + 1e-12)), r
        errs.append(float(np.max(err / absprod)))
    # wider inner ranges cost accuracy: more than 2^10 between r = 0 and r = 18
    assert errs[-1] > 2.0 ** 10 * errs[0], errs
    assert errs[0] < errs[2] < errs[3], errs
