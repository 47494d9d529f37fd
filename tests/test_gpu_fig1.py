"""Fig. 1 of the paper through the GPU path: HPL-style data, growing n.

Section 6 reports that on A, b ~ U(-1/2, 1/2) (the HPL generator) the LU
solve with 6 INT8 splits fails the bar of 16 on the scaled residual of Eq. 8
while 7 splits pass, for every size of its sweep (the plotted values are not
in the text, only this outcome).  Checked here for n = 256 .. 4096 (the sizes
are not stated; this range spans the figure's qualitative claim), with the
oracle's residual of the same method beside the small sizes.
"""
import numpy as np
import pytest

from oracle import lu as olu, residual
from paper_2509_23565_gb300 import inputs
from paper_2509_23565_gb300.binding import ColMajor

pytestmark = pytest.mark.gpu


def _gpu_eq8(gpu_lib, A, b, nb, s):
    n = A.shape[0]
    dA = ColMajor.from_numpy(A)
    ipiv, info = gpu_lib.dgetrf(dA, nb=nb, slices=s)
    x = ColMajor.from_numpy(b.reshape(n, 1))
    gpu_lib.dgetrs(dA, ipiv, x)
    gpu_lib.sync_status()
    assert int(info.item()) == 0
    return residual.scaled_residual(A, x.numpy().ravel(), b)


@pytest.mark.parametrize("n", [256, 512, 1024, 2048, 4096])
def test_six_splits_fail_seven_pass(gpu_lib, n):
    A = inputs.uniform(n, n, seed=n, lo=-0.5, hi=0.5)
    b = inputs.vector(n, seed=n + 1, lo=-0.5, hi=0.5)
    nb = 64 if n <= 512 else 128
    r6 = _gpu_eq8(gpu_lib, A, b, nb, 6)
    r7 = _gpu_eq8(gpu_lib, A, b, nb, 7)
    assert r6 > 16 and r7 < 16, (n, r6, r7)
    # one more slice gains about 2^7 in the residual
    assert r6 / r7 > 30, (n, r6, r7)
    if n <= 512:
        # the oracle runs the same method: the same order of magnitude
        for s, g in ((6, r6), (7, r7)):
            LU, piv, _ = olu.getrf(A, nb=nb, update="emulated", s=s)
            o = residual.scaled_residual(A, olu.getrs(LU, piv, b), b)
            assert o / 4 < g < o * 4, (n, s, g, o)
