"""GPU LU / Cholesky / solves through the C-ABI, checked against the oracle.

Pivot order may legitimately differ between the emulated and the FP64
factorization (Section 4: only the Schur update is emulated, but its low-order
bits steer later pivot choices), so factorizations are compared through what is
unique: the factorization residual, the Eq. 8 scaled residual and backward
error of the solve (computed by the oracle on the CPU), exact results on
small-integer matrices (where every emulated product is exact), the info
index of singular / non-SPD inputs, and valid pivot vectors.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import lu as olu, residual
from paper_2509_23565_gb300 import inputs
from paper_2509_23565_gb300.binding import NB_AUTO, ColMajor, EmulError

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _factor(gpu_lib, A, nb, s, ld=None):
    dA = ColMajor.from_numpy(A, ld=ld)
    ipiv, info = gpu_lib.dgetrf(dA, nb=nb, slices=s)
    gpu_lib.sync_status()
    return dA, ipiv, int(info.item())


def _valid_ipiv(ipiv, n):
    p = ipiv.cpu().numpy()
    return p.shape == (n,) and (p >= np.arange(1, n + 1)).all() and (p <= n).all()


@pytest.mark.parametrize("n,nb", [(1, 64), (5, 16), (100, 32), (257, 64), (700, 128), (1024, 64), (1100, 256),
                                  (600, 384), (1100, 512), (1300, 512)])
@pytest.mark.parametrize("s", [7, 8])
def test_getrf_getrs_uniform(gpu_lib, n, nb, s):
    """Ragged sizes and every block size; panels wider than 256 columns are
    factored as two halves (384 = 256 + 128; n = 1100 at nb = 512 ends with a
    76-column panel, n = 1300 with 276 = 256 + 20)."""
    A = inputs.uniform(n, n, seed=10 + n)
    b = inputs.vector(n, seed=20 + n)
    dA, ipiv, info = _factor(gpu_lib, A, nb, s, ld=n + 2)
    assert info == 0 and _valid_ipiv(ipiv, n)
    LU = dA.numpy()
    # s = 8 reaches FP64-level factors; at s = 7 each emulated update carries
    # about 2^-42 k of relative error, so the factor residual is O(10) (the
    # oracle's emulated LU gives 12.6 at n = 257), while the solve still passes
    assert residual.lu_residual(A, LU, ipiv.cpu().numpy()) < (16 if s == 8 else 100)
    db = ColMajor.from_numpy(b)
    gpu_lib.dgetrs(dA, ipiv, db)
    gpu_lib.sync_status()
    x = db.numpy()[:, 0]
    assert residual.scaled_residual(A, x, b) < 16
    assert residual.backward_error(A, x, b) < 16
    # the device residual kernel agrees with the oracle's formula
    out = gpu_lib.backward_error(ColMajor.from_numpy(A), db, ColMajor.from_numpy(b)).cpu().numpy()
    assert abs(out[0] - residual.scaled_residual(A, x, b)) <= 1e-9 * max(1.0, out[0])
    assert abs(out[1] - residual.backward_error(A, x, b)) <= 1e-9 * max(1.0, out[1])


@pytest.mark.parametrize("r", [4, 8, 16])
@pytest.mark.parametrize("s", [7, 8])
def test_getrf_log_scaled(gpu_lib, r, s):
    n = 512
    A = inputs.log_scaled(n, n, r, seed=30 + r)
    b = inputs.vector(n, seed=31)
    dA, ipiv, info = _factor(gpu_lib, A, 64, s)
    assert info == 0
    db = ColMajor.from_numpy(b)
    gpu_lib.dgetrs(dA, ipiv, db)
    x = db.numpy()[:, 0]
    assert residual.backward_error(A, x, b) < 16


def test_emulation_quality_tracks_oracle(gpu_lib):
    """Same method on both sides: the GPU and oracle emulated LU give backward
    errors of the same order at every slice count (3 fails, 8 passes)."""
    n = 256
    A = inputs.uniform(n, n, seed=41)
    b = inputs.vector(n, seed=42)
    for s in (3, 5, 8):
        dA, ipiv, _ = _factor(gpu_lib, A, 64, s)
        db = ColMajor.from_numpy(b)
        gpu_lib.dgetrs(dA, ipiv, db)
        g = residual.backward_error(A, db.numpy()[:, 0], b)
        LU, piv, _ = olu.getrf(A, nb=64, update="emulated", s=s)
        o = residual.backward_error(A, olu.getrs(LU, piv, b), b)
        assert o / 30 < g < o * 30, (s, g, o)
        if s == 3:
            assert g > 16
        if s == 8:
            assert g < 16


@pytest.mark.parametrize("n", [16, 40, 60])
def test_wilkinson_growth_exact(gpu_lib, n):
    """Integer entries: every emulated product is exact, so the factors equal
    the FP64 ones and max|U| = 2^(n-1) exactly (Section 5)."""
    A = inputs.wilkinson(n)
    dA, ipiv, info = _factor(gpu_lib, A, 16, 7)
    assert info == 0
    LU = dA.numpy()
    assert (ipiv.cpu().numpy() == np.arange(1, n + 1)).all()
    assert np.abs(np.triu(LU)).max() == 2.0 ** (n - 1)
    LUo, _, _ = olu.getrf(A, nb=16)
    assert np.array_equal(LU, LUo)


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(Fraction(t)) for t in line.split()])
    return np.array(rows)


@pytest.mark.parametrize("name,A", [
    ("eq10_turing_inverse.txt", inputs.turing(5)),
    ("eq11_fibonacci_inverse.txt", inputs.parawilk(5, 2, 2, 0.0)),
    ("eq13_blocked_inverse.txt", inputs.parawilk(5, 5, 2, 1.0)),
])
def test_worked_inverses(gpu_lib, name, A):
    dA, ipiv, info = _factor(gpu_lib, A, 16, 7)
    assert info == 0
    dB = ColMajor.from_numpy(np.eye(5))
    gpu_lib.dgetrs(dA, ipiv, dB)
    assert np.abs(dB.numpy() - _golden(name)).max() <= 1e-15


def test_singular_info(gpu_lib):
    n = 200
    A = inputs.uniform(n, n, seed=50)
    A[:, 77] = 0.0
    _, _, info = _factor(gpu_lib, A, 32, 7)
    assert info == 78


def test_multiple_rhs(gpu_lib):
    n, nrhs = 300, 5
    A = inputs.uniform(n, n, seed=60)
    B = inputs.uniform(n, nrhs, seed=61)
    dA, ipiv, _ = _factor(gpu_lib, A, 64, 8)
    dB = ColMajor.from_numpy(B, ld=n + 3)
    gpu_lib.dgetrs(dA, ipiv, dB)
    X = dB.numpy()
    for j in range(nrhs):
        assert residual.backward_error(A, X[:, j], B[:, j]) < 16


@pytest.mark.parametrize("n,nrhs", [(700, 3), (1, 2), (257, 1), (600, 2)])
def test_interchanges_exact(gpu_lib, n, nrhs):
    """With unit factors (LU = I) the solve returns P B: the row interchanges
    alone, applied from gather maps of at most 256 interchanges each (several
    maps per call here) or, for one right-hand side, from the composite
    permutation.  Pivot rows repeat, fall inside and beyond each map's rows,
    and stay in place; the result must equal the interchanges applied one by
    one, bit for bit."""
    import torch
    rng = np.random.default_rng(70 + n)
    piv = np.empty(n, dtype=np.int32)
    hot = rng.integers(0, n, 4)                  # rows named by many interchanges
    for k in range(n):
        u = rng.random()
        if u < 0.2:
            p = k
        elif u < 0.5:
            p = max(k, int(hot[rng.integers(0, 4)]))
        else:
            p = int(rng.integers(k, n))
        piv[k] = p + 1
    B = inputs.uniform(n, nrhs, seed=71 + n)
    want = B.copy()
    for k in range(n):
        p = piv[k] - 1
        want[[k, p]] = want[[p, k]]
    dLU = ColMajor.from_numpy(np.eye(n))
    dB = ColMajor.from_numpy(B, ld=n + 1)
    gpu_lib.dgetrs(dLU, torch.from_numpy(piv).cuda(), dB)
    gpu_lib.sync_status()
    assert np.array_equal(dB.numpy(), want)


@pytest.mark.parametrize("n,nb,cond", [(130, 32, 1e2), (512, 64, 1e8), (1000, 128, 1e12), (1000, 256, 1e8),
                                       (333, 48, 1e4), (1100, 512, 1e8), (700, 320, 1e12)])
@pytest.mark.parametrize("s", [7, 8])
def test_potrf_potrs(gpu_lib, n, nb, cond, s):
    A = inputs.spd(n, cond, seed=70 + n)
    b = inputs.vector(n, seed=71)
    dA = ColMajor.from_numpy(A)
    info = gpu_lib.dpotrf(dA, nb=nb, slices=s)
    gpu_lib.sync_status()
    assert int(info.item()) == 0
    L = np.tril(dA.numpy())
    assert residual.chol_residual(A, L) < 16
    # the strictly upper triangle is left untouched
    assert np.array_equal(np.triu(dA.numpy(), 1), np.triu(A, 1))
    db = ColMajor.from_numpy(b)
    gpu_lib.dpotrs(dA, db)
    x = db.numpy()[:, 0]
    assert residual.backward_error(A, x, b) < 16


def test_potrs_multiple_rhs(gpu_lib):
    n, nrhs = 300, 4
    A = inputs.spd(n, 1e6, seed=75)
    B = inputs.uniform(n, nrhs, seed=76)
    dA = ColMajor.from_numpy(A)
    info = gpu_lib.dpotrf(dA, nb=64, slices=8)
    assert int(info.item()) == 0
    dB = ColMajor.from_numpy(B, ld=n + 5)
    gpu_lib.dpotrs(dA, dB)
    X = dB.numpy()
    for j in range(nrhs):
        assert residual.backward_error(A, X[:, j], B[:, j]) < 16


@pytest.mark.parametrize("nb,at", [(32, 150), (256, 300), (256, 45), (512, 390)])
def test_potrf_not_spd(gpu_lib, nb, at):
    """A negative diagonal entry makes the leading minor of that order
    non-positive; info is its 1-based index wherever it falls in the blocks
    and 32-column panels of the diagonal block."""
    A = inputs.spd(400, 10.0, seed=80)
    A[at, at] = -5.0
    dA = ColMajor.from_numpy(A)
    info = gpu_lib.dpotrf(dA, nb=nb, slices=7)
    assert int(info.item()) == at + 1


@pytest.mark.parametrize("n,nb", [(4096, 128), (4096, 512)])
def test_getrf_large_backward_error(gpu_lib, n, nb):
    A = inputs.uniform(n, n, seed=90)
    b = inputs.vector(n, seed=91)
    dA, ipiv, info = _factor(gpu_lib, A, nb, 7)
    assert info == 0 and _valid_ipiv(ipiv, n)
    db = ColMajor.from_numpy(b)
    gpu_lib.dgetrs(dA, ipiv, db)
    x = db.numpy()[:, 0]
    assert residual.backward_error(A, x, b) < 16


def test_autotune_nb(gpu_lib):
    """The block-size tuner picks from {128, 256, 512} (only 128 when one
    128-column panel covers n), keeps the choice, and nb = NB_AUTO factors
    with it (LU and Cholesky, checked by the oracle's residuals)."""
    assert gpu_lib.autotune_nb("lu", 100, 7) == 128
    n = 700
    nb = gpu_lib.autotune_nb("lu", n, 7)
    assert nb in (128, 256, 512)
    A = inputs.uniform(n, n, seed=95)
    b = inputs.vector(n, seed=96)
    dA = ColMajor.from_numpy(A)
    ipiv, info = gpu_lib.dgetrf(dA, nb=NB_AUTO, slices=7)
    assert int(info.item()) == 0 and _valid_ipiv(ipiv, n)
    assert residual.lu_residual(A, dA.numpy(), ipiv.cpu().numpy()) < 100
    db = ColMajor.from_numpy(b)
    gpu_lib.dgetrs(dA, ipiv, db)
    assert residual.backward_error(A, db.numpy()[:, 0], b) < 16
    # Cholesky: tuned on first use of NB_AUTO
    S = inputs.spd(600, 1e6, seed=97)
    dS = ColMajor.from_numpy(S)
    info = gpu_lib.dpotrf(dS, nb=NB_AUTO, slices=7)
    assert int(info.item()) == 0
    assert residual.chol_residual(S, np.tril(dS.numpy())) < 16
    assert gpu_lib.autotune_nb("chol", 600, 7) in (128, 256, 512)
    with pytest.raises(EmulError):
        gpu_lib.autotune_nb("lu", 0, 7)


def test_profile_phases(gpu_lib):
    """With profiling on, every phase of a factorization with more than one
    panel, and the solve, report device time (CUDA events)."""
    import torch
    n, nb = 1200, 128
    A = inputs.uniform(n, n, seed=91)
    b = inputs.vector(n, seed=92)
    gpu_lib.profile_read()
    gpu_lib.profile_enable(True)
    try:
        dA, ipiv, info = _factor(gpu_lib, A, nb, 7)
        x = ColMajor.from_numpy(b.reshape(n, 1))
        gpu_lib.dgetrs(dA, ipiv, x)
        torch.cuda.synchronize()
        prof = gpu_lib.profile_read()
    finally:
        gpu_lib.profile_enable(False)
    assert info == 0
    ph = prof["phase_ms"]
    for name in ("panel", "swap", "u12", "update", "solve"):
        assert ph[name] > 0.0, (name, ph)
    assert prof["product_launches"] > 0 and prof["kernel_launches"] > 0


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _gpu_scaled_residual(gpu_lib, A, b, nb, s):
    n = A.shape[0]
    dA, ipiv, info = _factor(gpu_lib, A, nb, s)
    x = ColMajor.from_numpy(b.reshape(n, 1))
    gpu_lib.dgetrs(dA, ipiv, x)
    gpu_lib.sync_status()
    return residual.scaled_residual(A, x.numpy().ravel(), b)


def test_table1_on_gpu(gpu_lib):
    """Table 1 through the GPU path: on ParaWilk_256(4, 15, 1/2) the scaled
    residual falls about two orders of magnitude per split and every value is
    within a factor 4 of the printed one (same generator family, another draw
    and library).  6 splits land at the bar of 16 (within a factor 2: 15.8 here,
    17.9 for the oracle on the same input, 39.1 printed), 7 splits are an order
    of magnitude below it."""
    paper = {r[0]: float(r[1]) for r in _golden_rows("table1_parawilk256.txt")}
    n = 256
    A = inputs.parawilk_random(n, 4, 15, 0.5, seed=256)
    b = inputs.vector(n, seed=257)
    res = [_gpu_scaled_residual(gpu_lib, A, b, 64, s) for s in (3, 4, 5, 6, 7, 8)]
    assert all(res[i] > res[i + 1] for i in range(len(res) - 1)), res
    assert 8 < res[3] < 32 and res[4] < 1.6, res
    for got, s in zip(res, (3, 4, 5, 6, 7, 8)):
        want = paper[str(s)]
        assert want / 4 < got < want * 4, (s, got, want)


def test_table2_parameters_on_gpu(gpu_lib):
    """All 15 rows of Table 2 (the first ParaWilk_n(d, b, 1) found to push the
    scaled residual of Eq. 8 past 16 at 6 and at 7 splits, n = 256..2048).
    The paper's parameters for 6 splits also push this emulation past 16 for
    n <= 640, within a factor 2 of the printed residual; for larger n they give
    2.6-16 here (printed 16.5-40.6).  Its parameters for 7 splits do not break
    this emulation anywhere: with the threshold t = s + 1, exact level sums and
    one final rounding, 7 splits stay below 16 (the printed 16-62 come from the
    library the paper measured).  In every row one more split lowers the
    residual by more than 10x (7 bits per split), and every 6-split residual is
    within a factor 16 of the printed one (same family, another random fill,
    another library)."""
    for row in _golden_rows("table2_parawilk.txt"):
        n, d6, b6, r6 = int(row[0]), int(row[1]), int(row[2]), float(row[3])
        d7, b7 = int(row[4]), int(row[5])
        bvec = inputs.vector(n, seed=n + 1)
        got6 = _gpu_scaled_residual(gpu_lib, inputs.parawilk_random(n, d6, b6, 1.0, seed=n), bvec, 64, 6)
        got7 = _gpu_scaled_residual(gpu_lib, inputs.parawilk_random(n, d7, b7, 1.0, seed=n), bvec, 64, 7)
        assert got7 < 16, (n, got7)
        assert r6 / 16 < got6 < r6 * 16, (n, got6, r6)
        if n <= 640:
            assert got6 > 16 and r6 / 2 < got6 < r6 * 2, (n, got6, r6)
        # the same family at 7 splits with the 6-split parameters: one split apart
        got67 = _gpu_scaled_residual(gpu_lib, inputs.parawilk_random(n, d6, b6, 1.0, seed=n), bvec, 64, 7)
        assert got6 > 10 * got67, (n, got6, got67)
