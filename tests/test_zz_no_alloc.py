"""The allocation-free emulated DGEMM against the regular entry point.

emul_dgemm_noalloc serves callers that cannot allocate device memory; it
keeps its scratch in a static device array.  Its results must be bit for bit
those of emul_dgemm, on two calls in a row (the second call reuses the array
the first one left behind), and sizes beyond the array must be refused.
"""
import ctypes

import numpy as np
import pytest

from paper_2509_23565_gb300 import inputs
from paper_2509_23565_gb300.binding import ColMajor, load

pytestmark = pytest.mark.gpu


def _noalloc():
    lib = load()
    fn = lib.emul_dgemm_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                   ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                   ctypes.c_int]
    return fn


def _call(fn, A, B, C, s, alpha, beta):
    import torch
    st = torch.cuda.current_stream().cuda_stream
    return fn(ctypes.c_void_p(st), C.m, C.n, A.n, alpha, ctypes.c_void_p(A.ptr), A.ld, ctypes.c_void_p(B.ptr), B.ld,
              beta, ctypes.c_void_p(C.ptr), C.ld, s)


def test_noalloc_matches_dgemm_twice(gpu_lib):
    import torch
    fn = _noalloc()
    cases = [(300, 260, 256, 7, -1.0, 1.0, 1), (129, 77, 1000, 8, 0.5, -2.0, 2)]
    for (m, n, k, s, alpha, beta, seed) in cases:
        A = inputs.log_scaled(m, k, 3, seed=seed)
        B = inputs.uniform(k, n, seed=seed + 10)
        C = inputs.uniform(m, n, seed=seed + 20)
        dA, dB = ColMajor.from_numpy(A), ColMajor.from_numpy(B)
        ref = ColMajor.from_numpy(C)
        gpu_lib.dgemm(dA, dB, ref, s, alpha, beta)
        got = ColMajor.from_numpy(C)
        assert _call(fn, dA, dB, got, s, alpha, beta) == 0
        torch.cuda.synchronize()
        gpu_lib.sync_status()
        r, g = ref.numpy(), got.numpy()
        assert np.array_equal(r.view(np.int64), g.view(np.int64))


def test_noalloc_matches_oracle(gpu_lib):
    """One call checked straight against the oracle's emulated product: the
    exact level sums rounded once, then C = RN(RN(alpha D) + RN(beta C))."""
    import torch
    from oracle import emulgemm
    fn = _noalloc()
    m, n, k, s, alpha, beta = 200, 170, 300, 7, -1.0, 1.0
    A = inputs.log_scaled(m, k, 4, seed=31)
    B = inputs.uniform(k, n, seed=32)
    C = inputs.uniform(m, n, seed=33)
    got = ColMajor.from_numpy(C)
    assert _call(fn, ColMajor.from_numpy(A), ColMajor.from_numpy(B), got, s, alpha, beta) == 0
    torch.cuda.synchronize()
    want = emulgemm.emul_gemm(A, B, s, alpha=alpha, beta=beta, C=C)
    assert np.array_equal(got.numpy().view(np.int64), want.view(np.int64))


def test_noalloc_rejects_oversize(gpu_lib):
    fn = _noalloc()
    m = n = 4096
    k = 512
    A = ColMajor.empty(m, k)
    B = ColMajor.empty(k, n)
    C = ColMajor.empty(m, n)
    assert _call(fn, A, B, C, 7, 1.0, 0.0) == -3      # EMUL_NO_WORKSPACE: beyond the 16 MiB scratch
