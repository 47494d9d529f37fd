"""Oracle of the learned slice selector (slice count per product block; the a-posteriori
check follows the validated error-free products the paper cites in Sec. 3).

* features(A, B): 32-bin histograms of the exponent offset of every entry from
  its row scale (A) and column scale (B): offset = e_row - E_entry, where E is
  the smallest E with |x| < 2^E; zero entries and offsets >= 31 fall in bin 31.
  Each histogram is divided by its entry count: 64 floats.
* slice_errors(A, B): for s = 3..8, max_ij |D_s - D_8|_ij / (4 k u (|A||B|)_ij),
  D_s the emulated product with s slices (oracle.emulgemm); entries with
  (|A||B|)_ij = 0 are skipped.  label = smallest s with error <= 1, else 8.
* MLP: 64 -> 128 -> 128 -> 128 -> 6, ReLU, softmax cross-entropy over the
  classes s = 3..8, weights rounded to BF16 for the forward pass (FP32/FP64
  arithmetic otherwise).  forward / backward in float64 for gradient checks.

Test infrastructure only (see the package docstring).
"""
import numpy as np

from . import emulgemm
from .split import NONFINITE, row_exponents

NBINS = 32
SIZES = (64, 128, 128, 128, 6)
U = 2.0 ** -53


def _entry_exponents(X):
    X = np.abs(np.asarray(X, dtype=np.float64))
    _, ex = np.frexp(X)
    return ex.astype(np.int64)


def _hist(X):
    """Histogram of row offsets of the rows of X (rows x k)."""
    X = np.asarray(X, dtype=np.float64)
    e = row_exponents(X)
    E = _entry_exponents(X)
    off = e[:, None] - E
    off = np.where(X == 0.0, NBINS - 1, off)
    off = np.clip(off, 0, NBINS - 1)
    valid = (e != NONFINITE)[:, None] & np.ones_like(off, dtype=bool)
    h = np.bincount(off[valid].ravel(), minlength=NBINS).astype(np.float64)
    tot = max(1, X.size)
    return h / tot


def features(A, B):
    return np.concatenate([_hist(A), _hist(np.asarray(B, dtype=np.float64).T)])


def slice_errors(A, B):
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    k = A.shape[1]
    D8 = emulgemm.emul_gemm(A, B, 8)
    scale = 4.0 * k * U * (np.abs(A) @ np.abs(B))
    ok = scale > 0
    out = []
    for s in range(3, 9):
        Ds = emulgemm.emul_gemm(A, B, s)
        out.append(float(np.max(np.abs(Ds - D8)[ok] / scale[ok])) if ok.any() else 0.0)
    return np.array(out)


def label_from_errors(err):
    for i, v in enumerate(err):
        if v <= 1.0:
            return 3 + i
    return 8


def bf16_round(x):
    """Round float32 values to BF16 (round to nearest even), returned as float64."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed):
    rng = np.random.default_rng(seed)
    params = []
    for i in range(len(SIZES) - 1):
        fan_in, fan_out = SIZES[i], SIZES[i + 1]
        W = rng.standard_normal((fan_out, fan_in)) * np.sqrt(2.0 / fan_in)
        params.append((W.astype(np.float32), np.zeros(fan_out, dtype=np.float32)))
    return params


def forward(params, X):
    """Returns (logits, cache) with the BF16-rounded weights."""
    h = np.asarray(X, dtype=np.float64)
    cache = []
    for i, (W, b) in enumerate(params):
        Wb = bf16_round(W)
        z = h @ Wb.T + b.astype(np.float64)
        cache.append((h, z, Wb))
        h = np.maximum(z, 0.0) if i < len(params) - 1 else z
    return h, cache


def loss_and_grads(params, X, labels):
    """Mean softmax cross-entropy over classes s = 3..8 and its gradients
    with respect to W (through the BF16 rounding, straight-through) and b."""
    logits, cache = forward(params, X)
    y = np.asarray(labels) - 3
    B = logits.shape[0]
    z = logits - logits.max(axis=1, keepdims=True)
    p = np.exp(z)
    p /= p.sum(axis=1, keepdims=True)
    loss = float(-np.mean(np.log(p[np.arange(B), y])))
    d = p.copy()
    d[np.arange(B), y] -= 1.0
    d /= B
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        h, zpre, Wb = cache[i]
        if i < len(params) - 1:
            d = d * (zpre > 0)
        gW = d.T @ h
        gb = d.sum(axis=0)
        grads[i] = (gW, gb)
        d = d @ Wb
    return loss, grads
