"""GPU parity of the emulated product against the oracle (through the C-ABI).

Slices and scales (Section 2, Eq. 1-4) and the INT32 level sums (Eq. 2) must
match bit for bit; the emulated DGEMM must match the oracle's exact-then-round
result bit for bit, for every alpha/beta form, ragged shapes, special values,
and at full size on sampled rows/columns (the row and column scales of a
sampled block are those of the full matrix, so the oracle's value of a sampled
entry is exact).
"""
import numpy as np
import pytest

from oracle import split, emulgemm
from paper_2509_23565_gb300 import inputs
from paper_2509_23565_gb300.binding import ColMajor, bf16_bits_to_int

pytestmark = pytest.mark.gpu


def _same_bits(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.array_equal(a.view(np.int64), b.view(np.int64))


def _special_matrix(m, n, seed):
    rng = np.random.default_rng(seed)
    A = inputs.log_scaled(m, n, 16, seed)
    flat = A.reshape(-1, order="F")
    picks = rng.choice(flat.size, size=min(flat.size, 12), replace=False)
    specials = [0.0, -0.0, 5e-324, -3e-320, 2.0**-1022, 1.7976931348623157e308, -1.0, 2.0**52 + 1, 1e-300,
                0.75, -2.0**-1000, 1.0 - 2**-53]
    for i, p in enumerate(picks):
        flat[p] = specials[i % len(specials)]
    return np.asfortranarray(flat.reshape((m, n), order="F"))


@pytest.mark.parametrize("m,k", [(1, 1), (7, 13), (130, 257), (64, 128), (300, 40)])
@pytest.mark.parametrize("s", [1, 3, 7, 8])
def test_split_rows_bitexact(gpu_lib, m, k, s):
    A = _special_matrix(m, k, seed=m * 1000 + k)
    if m > 3:
        A[2, min(1, k - 1)] = np.inf
        A[3, 0] = np.nan
        A[1, :] = 0.0
    exps, sl = gpu_lib.split(ColMajor.from_numpy(A), s, by="rows")
    e_ref, S_ref = split.split_rows(A, s)
    assert np.array_equal(exps.cpu().numpy().astype(np.int64), e_ref)
    got = bf16_bits_to_int(sl)
    ok = e_ref != split.NONFINITE
    assert np.array_equal(got[:, ok, :], S_ref[:, ok, :].astype(np.int64))
    assert (got[:, ~ok, :] == 0).all()


@pytest.mark.parametrize("k,n", [(1, 1), (13, 7), (257, 130), (128, 64)])
@pytest.mark.parametrize("s", [3, 7, 8])
def test_split_cols_bitexact(gpu_lib, k, n, s):
    B = _special_matrix(k, n, seed=k * 7 + n)
    exps, sl = gpu_lib.split(ColMajor.from_numpy(B, ld=k + 5), s, by="cols")
    f_ref, S_ref = split.split_cols(B, s)
    assert np.array_equal(exps.cpu().numpy().astype(np.int64), f_ref)
    assert np.array_equal(bf16_bits_to_int(sl), S_ref.astype(np.int64))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (5, 7, 3), (128, 128, 32), (200, 300, 100), (129, 257, 1000),
                                   (64, 64, 2100)])
@pytest.mark.parametrize("s", [3, 7, 8])
def test_level_sums_bitexact(gpu_lib, m, n, k, s):
    A = inputs.log_scaled(m, k, 4, seed=11 + m)
    B = inputs.uniform(k, n, seed=12 + n)
    got = gpu_lib.level_sums(ColMajor.from_numpy(A), ColMajor.from_numpy(B), s).cpu().numpy()
    _, SA = split.split_rows(A, s)
    _, SB = split.split_cols(B, s)
    want = emulgemm.level_sums(SA, SB, s + 1)
    for L in range(2, s + 2):
        assert np.array_equal(got[L - 2].T.astype(np.int64), want[L - 2]), f"level {L}"
    gpu_lib.sync_status()


@pytest.mark.parametrize("s,k", [(7, 128), (7, 256), (6, 224), (7, 1000), (8, 128), (8, 1040), (3, 2048)])
def test_level_sums_worst_case_magnitudes(gpu_lib, s, k):
    """Every digit 127 with one sign: each accumulator reaches its largest
    allowed magnitude (k * pairs * 127^2 up to 1040 * 127^2 < 2^24)."""
    m = n = 128
    A = np.full((m, k), 1.0 - 2.0**-53, order="F")
    B = np.full((k, n), -(1.0 - 2.0**-53), order="F")
    got = gpu_lib.level_sums(ColMajor.from_numpy(A), ColMajor.from_numpy(B), s).cpu().numpy()
    _, SA = split.split_rows(A, s)
    _, SB = split.split_cols(B, s)
    want = emulgemm.level_sums(SA, SB, s + 1)
    for L in range(2, s + 2):
        assert np.array_equal(got[L - 2].T.astype(np.int64), want[L - 2]), f"level {L}"
    gpu_lib.sync_status()


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (33, 17, 5), (128, 128, 128), (257, 129, 96), (200, 380, 300),
                                   (130, 70, 1500), (256, 200, 256), (130, 140, 192), (64, 300, 160)])
@pytest.mark.parametrize("s", [3, 6, 7, 8])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0), (0.5, -2.0)])
def test_dgemm_bitexact(gpu_lib, m, n, k, s, alpha, beta):
    A = inputs.log_scaled(m, k, 2, seed=m + 3 * k)
    B = inputs.uniform(k, n, seed=n + 5 * k)
    C = inputs.uniform(m, n, seed=m + n)
    if beta == 0.0:
        C[:] = np.nan          # C must not be read when beta == 0
    dC = ColMajor.from_numpy(C, ld=m + 3)
    gpu_lib.dgemm(ColMajor.from_numpy(A, ld=m + 1), ColMajor.from_numpy(B), dC, s, alpha, beta)
    gpu_lib.sync_status()
    want = emulgemm.emul_gemm(A, B, s, alpha=alpha, beta=beta, C=C)
    got = dC.numpy()
    assert _same_bits(got, want), np.nanmax(np.abs(got - want))


@pytest.mark.parametrize("s,k", [(7, 256), (7, 200), (6, 256), (5, 128), (8, 256)])
def test_dgemm_large_horner_state(gpu_lib, s, k):
    """Rows and columns whose digits are all near 127 with one sign drive the
    exact sum T to its largest magnitude (beyond 2^64 at s = 7, k = 256), which
    the epilogue rounds on its wide path; other rows are random, so one warp
    mixes both paths.  Bit for bit against the oracle, C - A B form."""
    m, n = 200, 170
    A = inputs.uniform(m, k, seed=31 + k)
    B = inputs.uniform(k, n, seed=32 + k)
    A[::3, :] = 1.0 - 2.0**-53                 # every third row: all digits 127
    B[:, ::2] = -(1.0 - 2.0**-53)              # every second column: all digits 127, other sign
    A[7, :] = -(1.0 - 2.0**-53)
    C = inputs.uniform(m, n, seed=33)
    dC = ColMajor.from_numpy(C)
    gpu_lib.dgemm(ColMajor.from_numpy(A), ColMajor.from_numpy(B), dC, s, -1.0, 1.0)
    gpu_lib.sync_status()
    want = emulgemm.emul_gemm(A, B, s, alpha=-1.0, beta=1.0, C=C)
    assert _same_bits(dC.numpy(), want)


def test_dgemm_special_values(gpu_lib):
    m, n, k = 70, 40, 50
    A = _special_matrix(m, k, 5)
    B = _special_matrix(k, n, 6)
    A[4, 4] = np.nan
    B[7, 9] = -np.inf
    A[10, :] = 0.0
    C = inputs.uniform(m, n, seed=7)
    dC = ColMajor.from_numpy(C)
    gpu_lib.dgemm(ColMajor.from_numpy(A), ColMajor.from_numpy(B), dC, 7, -1.0, 1.0)
    want = emulgemm.emul_gemm(A, B, 7, alpha=-1.0, beta=1.0, C=C)
    got = dC.numpy()
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert _same_bits(got[ok], want[ok])


def test_dgemm_k_zero_and_empty(gpu_lib):
    C = inputs.uniform(9, 4, seed=1)
    dC = ColMajor.from_numpy(C)
    gpu_lib.dgemm(ColMajor.empty(9, 0), ColMajor.empty(0, 4), dC, 7, -1.0, 1.0)
    assert _same_bits(dC.numpy(), emulgemm.emul_gemm(np.zeros((9, 0)), np.zeros((0, 4)), 7, -1.0, 1.0, C))
    gpu_lib.dgemm(ColMajor.empty(0, 5), ColMajor.empty(5, 4), ColMajor.empty(0, 4), 7)


@pytest.mark.parametrize("size,s,r", [(4096, 7, 0), (4096, 8, 16), (8192, 6, 4)])
def test_dgemm_full_size_sampled(gpu_lib, size, s, r):
    """Full-size product, parity on 48 sampled rows x 48 sampled columns."""
    import torch
    m = n = k = size
    A = inputs.log_scaled(m, k, r, seed=901) if r else inputs.uniform(m, k, seed=901)
    B = inputs.log_scaled(k, n, r, seed=902) if r else inputs.uniform(k, n, seed=902)
    dA, dB = ColMajor.from_numpy(A), ColMajor.from_numpy(B)
    dC = ColMajor.empty(m, n)
    gpu_lib.dgemm(dA, dB, dC, s)
    gpu_lib.sync_status()
    rng = np.random.default_rng(size + s)
    rows = np.sort(np.concatenate([[0, m - 1], rng.choice(m, 46, replace=False)]))
    cols = np.sort(np.concatenate([[0, n - 1], rng.choice(n, 46, replace=False)]))
    got = dC.store[torch.as_tensor(cols, device="cuda")][:, torch.as_tensor(rows, device="cuda")].cpu().numpy().T
    want = emulgemm.emul_gemm(A[rows, :], B[:, cols], s)
    assert _same_bits(got, want)
