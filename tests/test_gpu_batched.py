"""Batched uneven solves with reduced-slice factorization and FP64 refinement
(one persistent launch), checked with the oracle's residual measures."""
import json
import os

import numpy as np
import pytest

from oracle import residual
from paper_2509_23565_gb300 import inputs
from paper_2509_23565_gb300.binding import ColMajor

pytestmark = pytest.mark.gpu


def _systems(sizes, r, seed):
    As, bs = [], []
    for i, n in enumerate(sizes):
        A = inputs.log_scaled(n, n, r, seed=seed + i) if r else inputs.uniform(n, n, seed=seed + i)
        As.append(A)
        bs.append(inputs.vector(n, seed=seed + 1000 + i))
    return As, bs


@pytest.mark.parametrize("r,slices", [(0, 3), (0, 4), (8, 3), (8, 8)])
def test_batched_backward_error(gpu_lib, r, slices):
    sizes = [1, 2, 5, 64, 100, 257, 300] + list(inputs.batch_sizes(25, 16, 400, seed=7))
    As, bs = _systems(sizes, r, 100 + slices)
    dA = [ColMajor.from_numpy(A, ld=A.shape[0] + 1) for A in As]
    db = [ColMajor.from_numpy(b) for b in bs]
    info, berr, iters = gpu_lib.dgesv_batched_ir(dA, db, max_iter=20, slices=slices, nb=32)
    gpu_lib.sync_status()
    info, berr, iters = info.cpu().numpy(), berr.cpu().numpy(), iters.cpu().numpy()
    for i, (A, b) in enumerate(zip(As, bs)):
        x = db[i].numpy()[:, 0]
        assert info[i] == 0
        be = residual.backward_error(A, x, b)
        assert be <= 16, (i, A.shape[0], be, berr[i], iters[i])
        assert berr[i] <= 16          # the device's own FP64 residual estimate
        assert np.array_equal(dA[i].numpy(), A)          # A is not modified
    assert iters.max() <= 20
    if r == 0:
        # the reduced-slice factors are good preconditioners on U(-1, 1) data:
        # refinement gains ~7 s - 1 bits per step (a wrong level sum would show here)
        assert iters.max() <= 6, iters


def test_batched_config5_sample(gpu_lib):
    """A sample of the config-5 batch: n log-uniform in [64, 1024], half with r = 8."""
    sizes = inputs.batch_sizes(24, 64, 1024, seed=77)
    As, bs = [], []
    for i, n in enumerate(sizes):
        n = int(n)
        As.append(inputs.log_scaled(n, n, 8, seed=300 + i) if i % 2 else inputs.uniform(n, n, seed=300 + i))
        bs.append(inputs.vector(n, seed=600 + i))
    db = [ColMajor.from_numpy(b) for b in bs]
    info, berr, iters = gpu_lib.dgesv_batched_ir([ColMajor.from_numpy(A) for A in As], db, max_iter=30)
    for i, (A, b) in enumerate(zip(As, bs)):
        assert residual.backward_error(A, db[i].numpy()[:, 0], b) <= 16, i


def test_batched_singular_info(gpu_lib):
    As, bs = _systems([50, 80], 0, 5)
    As[1][:, 10] = 0.0
    info, _, _ = gpu_lib.dgesv_batched_ir([ColMajor.from_numpy(A) for A in As], [ColMajor.from_numpy(b) for b in bs],
                                          max_iter=5, slices=3, nb=16)
    info = info.cpu().numpy()
    assert info[0] == 0 and info[1] > 0


def test_autotune_cache_roundtrip(gpu_lib, tmp_path):
    path = str(tmp_path / "tune.json")
    gpu_lib.autotune(path)
    text = open(path).read()
    rows = json.loads(text)
    assert len(rows) == 4 and all(r["nb"] in (16, 32, 64) and r["s"] in (3, 4) for r in rows)
    gpu_lib.autotune(path)            # reads the cache
    As, bs = _systems([70, 200, 600], 0, 9)
    db = [ColMajor.from_numpy(b) for b in bs]
    info, berr, _ = gpu_lib.dgesv_batched_ir([ColMajor.from_numpy(A) for A in As], db, max_iter=20)
    for i, (A, b) in enumerate(zip(As, bs)):
        assert residual.backward_error(A, db[i].numpy()[:, 0], b) <= 16
