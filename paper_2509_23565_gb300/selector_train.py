"""Training driver of the slice selector (slice count per product block).

Tuples (features, label) are generated by the method itself on the GPU: for a
random product block drawn from the dynamic-range generators (u 10^e, e in
[-r, r], r in {0, 4, 8, 16}; m = n in {128, ..., 512}; k in {128, 256}) the
library computes the exponent-histogram features and, from one level-sum pass,
the error of the emulated product at every slice count; the label is the
fewest slices whose error stays within 4 k u (|A||B|)_ij.  The network is then
trained with the library's forward / backward / AdamW kernels.  This module
only orchestrates calls to the C-ABI.

    python -m paper_2509_23565_gb300.selector_train --tuples 200000 --out selector_weights.bin
"""
import argparse
import json
import os
import time

import numpy as np

from . import inputs
from .binding import ColMajor, Emul

SIZES = (128, 192, 256, 384, 512)
KS = (128, 256)
RANGES = (0, 4, 8, 16)


LU_N = 2048
LU_RANGES = (0, 1, 2, 4, 8, 16)


def _lu_blocks(lib, gen, rng):
    """(L21, U12) pairs of every step of one emulated LU (s = 8) of a generator matrix:
    the blocks the trailing updates of a factorization actually multiply."""
    import torch
    n = LU_N
    nb = int(rng.choice(KS))
    r = int(rng.choice(LU_RANGES))
    W = ColMajor(inputs.log_scaled_device(n, n, r, gen), n, n)
    lib.dgetrf(W, nb=nb, slices=8)
    out = []
    for j0 in range(0, n - nb, nb):
        L21 = W.store[j0:j0 + nb, j0 + nb:]               # columns j0.. of L below the block
        U12 = W.store[j0 + nb:, j0:j0 + nb]               # rows j0..j0+nb of U right of the block
        out.append((L21, U12, n - j0 - nb, nb))
    return out


def generate(lib, count, seed):
    """Half of the tuples from raw generator blocks, half from sub-blocks of the
    L and U factors of emulated LU factorizations of generator matrices."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed)
    X = torch.zeros((count, 64), dtype=torch.float32, device="cuda")
    E = torch.zeros((count, 6), dtype=torch.float64, device="cuda")
    pool = []
    for i in range(count):
        if i % 2 == 0:
            m = int(rng.choice(SIZES))
            k = int(rng.choice(KS))
            r = int(rng.choice(RANGES))
            A = ColMajor(inputs.log_scaled_device(m, k, r, gen), m, k)
            B = ColMajor(inputs.log_scaled_device(k, m, r, gen), k, m)
        else:
            if not pool:
                pool = _lu_blocks(lib, gen, rng)
            L21s, U12s, m2, k = pool.pop(int(rng.integers(len(pool))))
            m = min(m2, int(rng.choice(SIZES)))
            r0 = int(rng.integers(0, m2 - m + 1))
            c0 = int(rng.integers(0, m2 - m + 1))
            A = ColMajor(L21s[:, r0:r0 + m].contiguous(), m, k)      # rows r0.. of L21 (column-major store k x m)
            B = ColMajor(U12s[c0:c0 + m, :].contiguous(), k, m)      # columns c0.. of U12
        X[i] = lib.selector_features(A, B)
        E[i] = lib.slice_errors(A, B)
    lib.sync_status()
    ok = E <= 1.0
    first = torch.where(ok.any(dim=1), ok.float().argmax(dim=1), torch.full((count,), 5, device="cuda"))
    labels = (first + 3).to(torch.int32)
    return X, labels, E


def init_params(seed):
    """He-normal weights, zero biases, in the flat layout of the C-ABI."""
    rng = np.random.default_rng(seed)
    sizes = (64, 128, 128, 128, 6)
    parts = []
    for i in range(4):
        fan_in, fan_out = sizes[i], sizes[i + 1]
        parts.append((rng.standard_normal((fan_out, fan_in)) * np.sqrt(2.0 / fan_in)).astype(np.float32).ravel())
        parts.append(np.zeros(fan_out, dtype=np.float32))
    return np.concatenate(parts)


def train(lib, X, labels, epochs=30, batch=4096, lr=2e-3, wd=1e-4, seed=0):
    import torch
    lib.selector_set_params(init_params(seed))
    n = X.shape[0]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen, device="cuda")
        tot = 0.0
        nb = 0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            xb = X[idx].contiguous()
            yb = labels[idx].contiguous()
            lib.selector_train_step(xb, yb, lr, wd, loss)
            tot += float(loss.item())
            nb += 1
        hist.append(tot / max(1, nb))
    return hist


def evaluate(lib, X, labels):
    pred = []
    for b0 in range(0, X.shape[0], 8192):
        pred.append(lib.selector_predict(X[b0:b0 + 8192].contiguous()))
    import torch
    p = torch.cat(pred)
    acc = float((p == labels).float().mean())
    safe = float((p >= labels).float().mean())
    mean_pred = float(p.float().mean())
    return {"accuracy": acc, "not_below_label": safe, "mean_predicted_slices": mean_pred,
            "mean_label": float(labels.float().mean())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tuples", type=int, default=200000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--seed", type=int, default=4000)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "selector_weights.bin"))
    args = ap.parse_args()
    import torch
    lib = Emul()
    t0 = time.time()
    X, y, E = generate(lib, args.tuples, args.seed)
    t_gen = time.time() - t0
    n_tr = int(0.9 * args.tuples)
    t0 = time.time()
    hist = train(lib, X[:n_tr], y[:n_tr], epochs=args.epochs, seed=args.seed)
    t_tr = time.time() - t0
    rep = {"tuples": args.tuples, "gen_s": t_gen, "train_s": t_tr, "loss_first": hist[0], "loss_last": hist[-1],
           "train": evaluate(lib, X[:n_tr], y[:n_tr]), "heldout": evaluate(lib, X[n_tr:], y[n_tr:]),
           "label_counts": {str(s): int((y == s).sum()) for s in range(3, 9)}}
    lib.selector_save(args.out)
    print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()
