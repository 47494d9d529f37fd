"""GPU parity of the emulated product with the truncation threshold as a
parameter (Section 2, Eq. 2: the slice pairs kept are those with p + q <= t).

emul_dgemm_threshold must equal the oracle's emul_gemm(..., t=t) bit for bit
for thresholds below, at and above the method's t = s + 1, up to the full
s^2-pair product t = 2s; t = s + 1 must reproduce emul_dgemm; a threshold
outside 2..2s, or one whose 128-bit exact sum could overflow at this k, is
refused on the host before any launch.
"""
import numpy as np
import pytest

from oracle import emulgemm
from paper_2509_23565_gb300 import inputs
from paper_2509_23565_gb300.binding import ColMajor, EmulError

pytestmark = pytest.mark.gpu


def _same_bits(a, b):
    return np.array_equal(np.asarray(a, dtype=np.float64).view(np.int64), np.asarray(b, dtype=np.float64).view(np.int64))


def _run(gpu_lib, A, B, C, s, t, alpha, beta):
    dC = ColMajor.from_numpy(C, ld=C.shape[0] + 2)
    gpu_lib.dgemm(ColMajor.from_numpy(A, ld=A.shape[0] + 1), ColMajor.from_numpy(B), dC, s, alpha, beta, t=t)
    gpu_lib.sync_status()
    return dC.numpy()


@pytest.mark.parametrize("s,t", [(1, 2), (3, 2), (3, 6), (5, 3), (6, 4), (6, 9), (7, 10), (7, 13), (7, 14),
                                 (8, 12), (8, 16)])
@pytest.mark.parametrize("m,n,k", [(257, 129, 96), (130, 70, 1500), (200, 380, 300)])
def test_threshold_bitexact(gpu_lib, s, t, m, n, k):
    A = inputs.log_scaled(m, k, 2, seed=m + 7 * k)
    B = inputs.uniform(k, n, seed=n + 11 * k)
    C = inputs.uniform(m, n, seed=m + n + t)
    got = _run(gpu_lib, A, B, C, s, t, -1.0, 1.0)
    want = emulgemm.emul_gemm(A, B, s, alpha=-1.0, beta=1.0, C=C, t=t)
    assert _same_bits(got, want), np.nanmax(np.abs(got - want))


@pytest.mark.parametrize("s,t", [(4, 8), (7, 9)])
def test_threshold_general_alpha_beta(gpu_lib, s, t):
    m, n, k = 150, 90, 200
    A, B = inputs.uniform(m, k, seed=61), inputs.log_scaled(k, n, 8, seed=62)
    C = inputs.uniform(m, n, seed=63)
    got = _run(gpu_lib, A, B, C, s, t, 0.5, -2.0)
    assert _same_bits(got, emulgemm.emul_gemm(A, B, s, alpha=0.5, beta=-2.0, C=C, t=t))
    C[:] = np.nan            # beta == 0: C is not read
    got = _run(gpu_lib, A, B, C, s, t, 1.0, 0.0)
    assert _same_bits(got, emulgemm.emul_gemm(A, B, s, t=t))


@pytest.mark.parametrize("s", [3, 7])
def test_default_threshold_is_method(gpu_lib, s):
    m, n, k = 140, 130, 256
    A, B = inputs.uniform(m, k, seed=71), inputs.uniform(k, n, seed=72)
    C = np.zeros((m, n), order="F")
    ref = ColMajor.from_numpy(C)
    gpu_lib.dgemm(ColMajor.from_numpy(A), ColMajor.from_numpy(B), ref, s)
    got = _run(gpu_lib, A, B, C, s, s + 1, 1.0, 0.0)
    assert _same_bits(got, ref.numpy())


def test_threshold_error_decreases_to_full_product(gpu_lib):
    """Entries of 7s - 1 significant bits below a unit row / column scale: the
    split truncates nothing, so t = 2s gives the correctly rounded product and
    each lower threshold is no more accurate than the next."""
    s, m, n, k = 3, 64, 48, 40
    rng = np.random.default_rng(81)
    bits = 7 * s - 1
    A = np.asfortranarray(np.ldexp(rng.integers(-(2**bits), 2**bits, (m, k)).astype(np.float64), -bits))
    B = np.asfortranarray(np.ldexp(rng.integers(-(2**bits), 2**bits, (k, n)).astype(np.float64), -bits))
    A[:, 0] = 0.5 + 2.0**-bits
    B[0, :] = -(0.5 + 2.0**-bits)
    want = emulgemm.emul_gemm(A, B, s, t=2 * s)
    errs = []
    for t in range(2, 2 * s + 1):
        got = _run(gpu_lib, A, B, np.zeros((m, n), order="F"), s, t, 1.0, 0.0)
        assert _same_bits(got, emulgemm.emul_gemm(A, B, s, t=t))
        errs.append(float(np.max(np.abs(got - want))))
    assert errs[-1] == 0.0 and all(a >= b for a, b in zip(errs, errs[1:])), errs


def test_threshold_full_size_sampled(gpu_lib):
    """s = 7, t = 2s at 4096^3: parity on 40 sampled rows x 40 sampled columns."""
    import torch
    size, s, t = 4096, 7, 14
    A, B = inputs.uniform(size, size, seed=91), inputs.log_scaled(size, size, 4, seed=92)
    dC = ColMajor.empty(size, size)
    gpu_lib.dgemm(ColMajor.from_numpy(A), ColMajor.from_numpy(B), dC, s, t=t)
    gpu_lib.sync_status()
    rng = np.random.default_rng(93)
    rows = np.sort(np.concatenate([[0, size - 1], rng.choice(np.arange(1, size - 1), 38, replace=False)]))
    cols = np.sort(np.concatenate([[0, size - 1], rng.choice(np.arange(1, size - 1), 38, replace=False)]))
    got = dC.store[torch.as_tensor(cols, device="cuda")][:, torch.as_tensor(rows, device="cuda")].cpu().numpy().T
    assert _same_bits(got, emulgemm.emul_gemm(A[rows, :], B[:, cols], s, t=t))


def test_threshold_refused_on_host(gpu_lib):
    A, B, C = ColMajor.empty(4, 8), ColMajor.empty(8, 4), ColMajor.empty(4, 4)
    for s, t in ((4, 1), (4, 9), (7, 15)):
        with pytest.raises(EmulError, match="INVALID_ARG"):
            gpu_lib.dgemm(A, B, C, s, t=t)
    # s = 8, t = 16: the exact sum grows by about 2^112 per unit of k, so
    # k = 20000 could exceed 2^126 and is refused; k = 4096 is accepted
    A, B = ColMajor.empty(2, 20000), ColMajor.empty(20000, 2)
    with pytest.raises(EmulError, match="NOT_SUPPORTED"):
        gpu_lib.dgemm(A, B, ColMajor.empty(2, 2), 8, t=16)
    A = ColMajor.from_numpy(inputs.uniform(2, 4096, seed=5))
    B = ColMajor.from_numpy(inputs.uniform(4096, 2, seed=6))
    dC = ColMajor.empty(2, 2)
    gpu_lib.dgemm(A, B, dC, 8, t=16)
    gpu_lib.sync_status()
    assert _same_bits(dC.numpy(), emulgemm.emul_gemm(A.numpy(), B.numpy(), 8, t=16))



@pytest.mark.parametrize("sa,sb,t", [(3, 7, 0), (7, 3, 0), (5, 8, 0), (8, 2, 0), (4, 6, 10), (7, 7, 0),
                                     (6, 2, 8), (2, 7, 5)])
@pytest.mark.parametrize("m,n,k", [(130, 70, 96), (257, 129, 256), (64, 300, 160)])
def test_unequal_slices_bitexact(gpu_lib, sa, sb, t, m, n, k):
    """Unequal slice counts (pairs p <= sa, q <= sb, p + q <= t) bit for bit
    against the oracle, Schur-update form."""
    A = inputs.log_scaled(m, k, 3, seed=m + sa)
    B = inputs.uniform(k, n, seed=n + sb)
    C = inputs.uniform(m, n, seed=m + n + t)
    dC = ColMajor.from_numpy(C)
    gpu_lib.dgemm_unequal(ColMajor.from_numpy(A), ColMajor.from_numpy(B), dC, sa, sb, -1.0, 1.0, t)
    gpu_lib.sync_status()
    want = emulgemm.emul_gemm_unequal(A, B, sa, sb, alpha=-1.0, beta=1.0, C=C, t=t or None)
    assert np.array_equal(dC.numpy().view(np.int64), want.view(np.int64))


def test_unequal_rejects_bad_threshold(gpu_lib):
    A = ColMajor.empty(10, 10)
    with pytest.raises(Exception):
        gpu_lib.dgemm_unequal(A, A, ColMajor.empty(10, 10), 3, 2, 1.0, 0.0, 6)
