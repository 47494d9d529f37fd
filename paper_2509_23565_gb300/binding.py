"""Thin ctypes binding of the C-ABI library (include/emul.h).

Argument marshalling only: every step runs inside libemul.so.  Loading fails
loudly if the library has not been built (there is no fallback).  PyTorch is
used for device memory and streams.

Matrices cross the boundary in column-major order.  A column-major m x n matrix
with leading dimension ld is held here as a torch tensor `store` of shape
(n, ld) (row j of `store` is column j of the matrix); ``ColMajor`` wraps it.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libemul.so")

EMUL_OK = 0
NB_AUTO = -1          # EMUL_NB_AUTO: block size from emul_autotune_nb
STATUS = {0: "EMUL_OK", -1: "EMUL_INVALID_ARG", -2: "EMUL_CUDA_ERROR", -3: "EMUL_NO_WORKSPACE",
          -4: "EMUL_TIMEOUT", -5: "EMUL_NOT_SUPPORTED"}

# name -> (restype, argtypes); mirrors include/emul.h
_c_int, _c_long, _c_double, _vp, _c_char = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_void_p, ctypes.c_char
SIGNATURES = {
    "emul_create": (_c_int, [ctypes.POINTER(_vp), _vp]),
    "emul_destroy": (_c_int, [_vp]),
    "emul_set_stream": (_c_int, [_vp, _vp]),
    "emul_last_error": (ctypes.c_char_p, [_vp]),
    "emul_sync_status": (_c_int, [_vp]),
    "emul_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "emul_schedule": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_int, _vp, _c_int, _vp, _c_int, _vp]),
    "emul_split": (_c_int, [_vp, _c_int, _c_int, _vp, _c_long, _c_long, _c_int, _vp, _vp, _c_long]),
    "emul_level_sums": (_c_int, [_vp, _c_int, _c_int, _c_int, _vp, _c_int, _vp, _c_int, _c_int, _vp, _c_int,
                                 _c_long]),
    "emul_dgemm": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_double, _vp, _c_int, _vp, _c_int, _c_double, _vp,
                            _c_int, _c_int]),
    "emul_dgemm_threshold": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_double, _vp, _c_int, _vp, _c_int, _c_double,
                                      _vp, _c_int, _c_int, _c_int]),
    "emul_dgemm_unequal": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_double, _vp, _c_int, _vp, _c_int, _c_double,
                                    _vp, _c_int, _c_int, _c_int, _c_int]),
    "emul_dgetrf": (_c_int, [_vp, _c_int, _vp, _c_int, _vp, _c_int, _c_int, _vp, _vp]),
    "emul_dgetrf_nopiv": (_c_int, [_vp, _c_int, _vp, _c_int, _c_int, _c_int, _vp, _vp]),
    "emul_dgetrs": (_c_int, [_vp, _c_int, _c_int, _vp, _c_int, _vp, _vp, _c_int]),
    "emul_dpotrf": (_c_int, [_vp, _c_char, _c_int, _vp, _c_int, _c_int, _c_int, _vp, _vp]),
    "emul_dpotrs": (_c_int, [_vp, _c_char, _c_int, _c_int, _vp, _c_int, _vp, _c_int]),
    "emul_backward_error": (_c_int, [_vp, _c_int, _vp, _c_int, _vp, _vp, _vp]),
    "emul_selector_features": (_c_int, [_vp, _c_int, _c_int, _c_int, _vp, _c_int, _vp, _c_int, _vp]),
    "emul_slice_errors": (_c_int, [_vp, _c_int, _c_int, _c_int, _vp, _c_int, _vp, _c_int, _vp]),
    "emul_selector_set_params": (_c_int, [_vp, _vp]),
    "emul_selector_get_params": (_c_int, [_vp, _vp]),
    "emul_selector_grad": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _vp]),
    "emul_selector_train_step": (_c_int, [_vp, _c_int, _vp, _vp, ctypes.c_float, ctypes.c_float, _vp]),
    "emul_selector_predict": (_c_int, [_vp, _c_int, _vp, _vp]),
    "emul_selector_save": (_c_int, [_vp, ctypes.c_char_p]),
    "emul_selector_load": (_c_int, [_vp, ctypes.c_char_p]),
    "emul_dgesv_batched_ir": (_c_int, [_vp, _c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _c_int, _c_int, _c_int]),
    "emul_autotune": (_c_int, [_vp, ctypes.c_char_p]),
    "emul_autotune_nb": (_c_int, [_vp, _c_int, _c_int, _c_int, _vp]),
    "emul_profile_enable": (_c_int, [_vp, _c_int]),
    "emul_profile_read": (_c_int, [_vp, _vp]),
}

_LIB = None


class EmulError(RuntimeError):
    pass


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("slices_min", ctypes.c_int), ("slices_max", ctypes.c_int),
                ("checks_failed", ctypes.c_int), ("seconds", ctypes.c_double), ("slices_mean", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("product_launches", ctypes.c_longlong),
                ("product_ms", ctypes.c_double), ("product_tensor_flops", ctypes.c_double),
                ("product_bytes", ctypes.c_double), ("phase_ms", ctypes.c_double * 5)]

PHASES = ("panel", "swap", "u12", "update", "solve")   # EMUL_PHASE_* order


def load():
    """Load libemul.so and declare every exported signature (no CUDA call)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise EmulError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


class ColMajor:
    """Column-major m x n FP64 (or other dtype) matrix on the device."""

    def __init__(self, store, m, n):
        self.store, self.m, self.n = store, m, n
        self.ld = store.shape[1]

    @property
    def ptr(self):
        return self.store.data_ptr()

    @staticmethod
    def from_numpy(A, device="cuda", ld=None, dtype=None):
        import torch
        A = np.asarray(A)
        if A.ndim == 1:
            A = A[:, None]
        m, n = A.shape
        ld = m if ld is None else ld
        buf = np.zeros((n, max(ld, 1)), dtype=A.dtype if dtype is None else dtype)
        buf[:, :m] = A.T
        return ColMajor(torch.from_numpy(buf).to(device), m, n)

    @staticmethod
    def empty(m, n, device="cuda", ld=None, dtype=None):
        import torch
        ld = m if ld is None else ld
        return ColMajor(torch.zeros((n, max(ld, 1)), dtype=dtype or torch.float64, device=device), m, n)

    def numpy(self):
        return self.store[:, :self.m].cpu().numpy().T.copy()


class Emul:
    """One library handle bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream=None):
        import torch
        self.lib = load()
        self.h = _vp()
        st = (stream or torch.cuda.current_stream()).cuda_stream
        self._check(self.lib.emul_create(ctypes.byref(self.h), _vp(st)), "emul_create")

    def close(self):
        if self.h:
            self.lib.emul_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != EMUL_OK:
            msg = self.lib.emul_last_error(self.h).decode() if self.h else ""
            raise EmulError(f"{what}: {STATUS.get(rc, rc)} {msg}")

    def set_stream(self, stream):
        self._check(self.lib.emul_set_stream(self.h, _vp(stream.cuda_stream)), "emul_set_stream")

    def sync_status(self):
        self._check(self.lib.emul_sync_status(self.h), "emul_sync_status")

    def profile_enable(self, on=True):
        self._check(self.lib.emul_profile_enable(self.h, 1 if on else 0), "emul_profile_enable")

    def profile_read(self):
        p = Profile()
        self._check(self.lib.emul_profile_read(self.h, ctypes.byref(p)), "emul_profile_read")
        out = {k: getattr(p, k) for k, _ in Profile._fields_ if k != "phase_ms"}
        out["phase_ms"] = {name: float(p.phase_ms[i]) for i, name in enumerate(PHASES)}
        return out

    def workspace_bytes(self):
        return int(self.lib.emul_workspace_bytes(self.h))

    # ---------------------------------------------------------------- steps
    def split(self, X, slices, by="rows"):
        """Slices of a ColMajor operand by rows (A) or by columns (B).
        Returns (exps int32 [rows], slices int16 view of BF16 bits [s, rows, ldk])."""
        import torch
        if by == "rows":
            rows, k, rs, cs = X.m, X.n, 1, X.ld
        else:
            rows, k, rs, cs = X.n, X.m, X.ld, 1
        ldk = (k + 7) // 8 * 8
        exps = torch.zeros(max(rows, 1), dtype=torch.int32, device="cuda")
        out = torch.zeros((slices, max(rows, 1), max(ldk, 8)), dtype=torch.int16, device="cuda")
        self._check(self.lib.emul_split(self.h, rows, k, _vp(X.ptr), rs, cs, slices, _vp(exps.data_ptr()),
                                        _vp(out.data_ptr()), max(ldk, 8)), "emul_split")
        return exps[:rows], out[:, :rows, :k]

    def level_sums(self, A, B, slices):
        import torch
        m, k, n = A.m, A.n, B.n
        out = torch.zeros((slices, n, max(m, 1)), dtype=torch.int32, device="cuda")
        self._check(self.lib.emul_level_sums(self.h, m, n, k, _vp(A.ptr), A.ld, _vp(B.ptr), B.ld, slices,
                                             _vp(out.data_ptr()), max(m, 1), n * max(m, 1)), "emul_level_sums")
        return out   # out[L-2, j, i] = I_L(i, j)

    # ---------------------------------------------------------------- BLAS / LAPACK
    def dgemm(self, A, B, C, slices, alpha=1.0, beta=0.0, t=None):
        if t is None:
            self._check(self.lib.emul_dgemm(self.h, C.m, C.n, A.n, alpha, _vp(A.ptr), A.ld, _vp(B.ptr), B.ld, beta,
                                            _vp(C.ptr), C.ld, slices), "emul_dgemm")
        else:
            self._check(self.lib.emul_dgemm_threshold(self.h, C.m, C.n, A.n, alpha, _vp(A.ptr), A.ld, _vp(B.ptr),
                                                      B.ld, beta, _vp(C.ptr), C.ld, slices, t),
                        "emul_dgemm_threshold")

    def dgemm_unequal(self, A, B, C, slices_a, slices_b, alpha=1.0, beta=0.0, t=0):
        self._check(self.lib.emul_dgemm_unequal(self.h, C.m, C.n, A.n, alpha, _vp(A.ptr), A.ld, _vp(B.ptr), B.ld,
                                                beta, _vp(C.ptr), C.ld, slices_a, slices_b, t), "emul_dgemm_unequal")

    def autotune_nb(self, kind, n, slices=7):
        """Block size of emul_dgetrf (kind "lu") or emul_dpotrf ("chol") for n x n
        at `slices`, tuned over {128, 256, 512} and kept in the handle (nb=NB_AUTO
        then uses it)."""
        out = ctypes.c_int(0)
        k = {"lu": 0, "chol": 1}[kind]
        self._check(self.lib.emul_autotune_nb(self.h, k, n, slices, ctypes.byref(out)), "emul_autotune_nb")
        return out.value

    def dgetrf(self, A, nb=0, slices=7, stats=False):
        import torch
        ipiv = torch.zeros(max(A.m, 1), dtype=torch.int32, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = Stats()
        self._check(self.lib.emul_dgetrf(self.h, A.m, _vp(A.ptr), A.ld, _vp(ipiv.data_ptr()), nb, slices,
                                         _vp(info.data_ptr()), ctypes.byref(st)), "emul_dgetrf")
        return (ipiv[:A.m], info, st) if stats else (ipiv[:A.m], info)

    def dgetrf_nopiv(self, A, nb=0, slices=7, stats=False):
        """LU without pivoting; returns (ipiv = 1..n for dgetrs, info[, stats])."""
        import torch
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = Stats()
        self._check(self.lib.emul_dgetrf_nopiv(self.h, A.m, _vp(A.ptr), A.ld, nb, slices, _vp(info.data_ptr()),
                                               ctypes.byref(st)), "emul_dgetrf_nopiv")
        ipiv = torch.arange(1, A.m + 1, dtype=torch.int32, device="cuda")
        return (ipiv, info, st) if stats else (ipiv, info)

    def dgetrs(self, LU, ipiv, B):
        self._check(self.lib.emul_dgetrs(self.h, LU.m, B.n, _vp(LU.ptr), LU.ld, _vp(ipiv.data_ptr()), _vp(B.ptr),
                                         B.ld), "emul_dgetrs")

    def dpotrf(self, A, nb=0, slices=7, stats=False):
        import torch
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = Stats()
        self._check(self.lib.emul_dpotrf(self.h, b"L", A.m, _vp(A.ptr), A.ld, nb, slices, _vp(info.data_ptr()),
                                         ctypes.byref(st)), "emul_dpotrf")
        return (info, st) if stats else info

    def dpotrs(self, L, B):
        self._check(self.lib.emul_dpotrs(self.h, b"L", L.m, B.n, _vp(L.ptr), L.ld, _vp(B.ptr), B.ld),
                    "emul_dpotrs")

    # ---------------------------------------------------------------- batched
    def dgesv_batched_ir(self, As, bs, max_iter=10, slices=0, nb=0):
        """As: list of ColMajor n_i x n_i (not modified); bs: list of ColMajor n_i x 1
        (overwritten by x_i).  Returns (info, berr, iters) as device tensors."""
        import torch
        count = len(As)
        n_arr = (ctypes.c_int * count)(*[a.m for a in As])
        lda_arr = (ctypes.c_int * count)(*[a.ld for a in As])
        A_arr = (ctypes.c_void_p * count)(*[a.ptr for a in As])
        b_arr = (ctypes.c_void_p * count)(*[b.ptr for b in bs])
        info = torch.zeros(max(count, 1), dtype=torch.int32, device="cuda")
        berr = torch.zeros(max(count, 1), dtype=torch.float64, device="cuda")
        iters = torch.zeros(max(count, 1), dtype=torch.int32, device="cuda")
        self._check(self.lib.emul_dgesv_batched_ir(self.h, count, n_arr, A_arr, lda_arr, b_arr, _vp(info.data_ptr()),
                                                   _vp(berr.data_ptr()), _vp(iters.data_ptr()), max_iter, slices, nb),
                    "emul_dgesv_batched_ir")
        return info[:count], berr[:count], iters[:count]

    def autotune(self, cache_path=None):
        self._check(self.lib.emul_autotune(self.h, cache_path.encode() if cache_path else None), "emul_autotune")

    # ---------------------------------------------------------------- selector
    SELECTOR_PARAMS = 42118

    def selector_features(self, A, B):
        import torch
        feat = torch.zeros(64, dtype=torch.float32, device="cuda")
        self._check(self.lib.emul_selector_features(self.h, A.m, B.n, A.n, _vp(A.ptr), A.ld, _vp(B.ptr), B.ld,
                                                    _vp(feat.data_ptr())), "emul_selector_features")
        return feat

    def slice_errors(self, A, B):
        import torch
        err = torch.zeros(6, dtype=torch.float64, device="cuda")
        self._check(self.lib.emul_slice_errors(self.h, A.m, B.n, A.n, _vp(A.ptr), A.ld, _vp(B.ptr), B.ld,
                                               _vp(err.data_ptr())), "emul_slice_errors")
        return err

    def selector_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.SELECTOR_PARAMS
        self._check(self.lib.emul_selector_set_params(self.h, p.ctypes.data_as(_vp)), "emul_selector_set_params")

    def selector_get_params(self):
        p = np.zeros(self.SELECTOR_PARAMS, dtype=np.float32)
        self._check(self.lib.emul_selector_get_params(self.h, p.ctypes.data_as(_vp)), "emul_selector_get_params")
        return p

    def selector_grad(self, X, labels):
        import torch
        g = torch.zeros(self.SELECTOR_PARAMS, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self._check(self.lib.emul_selector_grad(self.h, X.shape[0], _vp(X.data_ptr()), _vp(labels.data_ptr()),
                                                _vp(g.data_ptr()), _vp(loss.data_ptr())), "emul_selector_grad")
        return g, loss

    def selector_train_step(self, X, labels, lr, weight_decay=0.0, loss=None):
        self._check(self.lib.emul_selector_train_step(self.h, X.shape[0], _vp(X.data_ptr()), _vp(labels.data_ptr()),
                                                      lr, weight_decay, _vp(loss.data_ptr() if loss is not None else 0)),
                    "emul_selector_train_step")

    def selector_predict(self, X):
        import torch
        out = torch.zeros(X.shape[0], dtype=torch.int32, device="cuda")
        self._check(self.lib.emul_selector_predict(self.h, X.shape[0], _vp(X.data_ptr()), _vp(out.data_ptr())),
                    "emul_selector_predict")
        return out

    def selector_save(self, path):
        self._check(self.lib.emul_selector_save(self.h, path.encode()), "emul_selector_save")

    def selector_load(self, path):
        self._check(self.lib.emul_selector_load(self.h, path.encode()), "emul_selector_load")

    def backward_error(self, A, x, b):
        import torch
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        self._check(self.lib.emul_backward_error(self.h, A.m, _vp(A.ptr), A.ld, _vp(x.ptr), _vp(b.ptr),
                                                 _vp(out.data_ptr())), "emul_backward_error")
        return out


SWEEP_FIELDS = ("k0c", "k1c", "L0", "L1", "pb0", "pb1", "pe0", "pe1", "flags0", "flags1", "nplanes", "kcs")


def schedule(slices, k, wide=False, level_sums=False, t=0):
    """Product-kernel schedule for (slices, k) and levels 2..t (t = 0:
    slices + 1) from emul_schedule (host only): (list of sweep dicts with
    SWEEP_FIELDS, slot table bytes, meta dict), or None when no schedule
    exists."""
    L = load()
    meta = (ctypes.c_int * 5)()
    rc = L.emul_schedule(slices, k, int(wide), int(level_sums), t, None, 0, None, 0, meta)
    if meta[0] == 0:
        return None
    sw = (ctypes.c_int * (meta[0] * len(SWEEP_FIELDS)))()
    tab = (ctypes.c_ubyte * max(1, meta[4]))()
    rc = L.emul_schedule(slices, k, int(wide), int(level_sums), t, sw, meta[0], tab, meta[4], meta)
    if rc != 0:
        raise EmulError(f"emul_schedule failed ({rc})")
    n = len(SWEEP_FIELDS)
    sweeps = [dict(zip(SWEEP_FIELDS, sw[i * n:(i + 1) * n])) for i in range(meta[0])]
    info = {"nsweeps": meta[0], "njobs": meta[1], "t0": meta[2], "period": meta[3], "table_bytes": meta[4]}
    return sweeps, bytes(tab[:meta[4]]), info


def lib():
    """A ready handle on torch's current stream (tests use one per session)."""
    return Emul()


def bf16_bits_to_int(t):
    """BF16 bit patterns (int16 tensor) of small integers -> int64 numpy values."""
    import torch
    f = t.view(torch.bfloat16).float().cpu().numpy()
    return f.astype(np.int64)
