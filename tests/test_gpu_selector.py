"""GPU slice selector against the oracle: features bit for bit, label errors,
MLP gradients (BF16 weights, FP32 accumulation), training, weights file, and
emul_dgetrf with slices = 0 (selector + a-posteriori probe)."""
import os

import numpy as np
import pytest

from oracle import lu as olu, residual, selector
from paper_2509_23565_gb300 import inputs
from paper_2509_23565_gb300.binding import ColMajor
from paper_2509_23565_gb300.selector_train import init_params

pytestmark = pytest.mark.gpu
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2509_23565_gb300",
                       "selector_weights.bin")


def _flat_to_layers(p):
    sizes = (64, 128, 128, 128, 6)
    out, o = [], 0
    for i in range(4):
        W = p[o:o + sizes[i + 1] * sizes[i]].reshape(sizes[i + 1], sizes[i])
        o += W.size
        b = p[o:o + sizes[i + 1]]
        o += b.size
        out.append((W, b))
    return out


@pytest.mark.parametrize("m,n,k,r", [(100, 70, 33, 0), (256, 300, 128, 8), (40, 512, 256, 16)])
def test_features_bitexact(gpu_lib, m, n, k, r):
    A = inputs.log_scaled(m, k, r, seed=m + k) if r else inputs.uniform(m, k, seed=m)
    B = inputs.log_scaled(k, n, r, seed=n + k) if r else inputs.uniform(k, n, seed=n)
    A[3, 2] = 0.0
    got = gpu_lib.selector_features(ColMajor.from_numpy(A), ColMajor.from_numpy(B)).cpu().numpy()
    want = selector.features(A, B).astype(np.float32)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("m,k,r", [(96, 128, 0), (130, 256, 4), (64, 128, 16)])
def test_slice_errors_match_oracle(gpu_lib, m, k, r):
    A = inputs.log_scaled(m, k, r, seed=1 + m) if r else inputs.uniform(m, k, seed=1 + m)
    B = inputs.log_scaled(k, m, r, seed=2 + m) if r else inputs.uniform(k, m, seed=2 + m)
    got = gpu_lib.slice_errors(ColMajor.from_numpy(A), ColMajor.from_numpy(B)).cpu().numpy()
    want = selector.slice_errors(A, B)
    assert np.allclose(got, want, rtol=1e-9, atol=0.0), (got, want)
    assert selector.label_from_errors(got) == selector.label_from_errors(want)


def test_gradients_match_oracle(gpu_lib):
    import torch
    rng = np.random.default_rng(3)
    p = init_params(11)
    gpu_lib.selector_set_params(p)
    X = rng.random((50, 64)).astype(np.float32)
    y = rng.integers(3, 9, 50).astype(np.int32)
    g, loss = gpu_lib.selector_grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    lo, go = selector.loss_and_grads(_flat_to_layers(p), X.astype(np.float64), y)
    assert abs(float(loss.item()) - lo) <= 1e-4 * abs(lo)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in go])
    gg = g.cpu().numpy().astype(np.float64)
    assert np.abs(gg - flat).max() <= 1e-4 * np.abs(flat).max() + 1e-7


def test_training_learns_and_roundtrips(gpu_lib, tmp_path):
    import torch
    from paper_2509_23565_gb300.selector_train import train, evaluate
    rng = np.random.default_rng(4)
    # separable synthetic task: label determined by where the feature mass lies
    n = 6000
    X = np.zeros((n, 64), dtype=np.float32)
    y = rng.integers(3, 9, n).astype(np.int32)
    for i in range(n):
        X[i, (y[i] - 3) * 5:(y[i] - 3) * 5 + 5] = rng.random(5)
        X[i, 32 + (y[i] - 3) * 4] = 1.0
    Xt, yt = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    hist = train(gpu_lib, Xt, yt, epochs=15, batch=1024, lr=3e-3, seed=5)
    assert hist[-1] < 0.3 * hist[0]
    assert evaluate(gpu_lib, Xt, yt)["accuracy"] > 0.95
    f = str(tmp_path / "w.bin")
    gpu_lib.selector_save(f)
    before = gpu_lib.selector_predict(Xt[:100].contiguous()).cpu().numpy()
    gpu_lib.selector_set_params(init_params(99))
    gpu_lib.selector_load(f)
    after = gpu_lib.selector_predict(Xt[:100].contiguous()).cpu().numpy()
    assert np.array_equal(before, after)


def test_auto_slices_lu(gpu_lib):
    """slices = 0: per-step choice by the selector, probe-checked; the solve
    meets the Eq. 8 bar and the statistics report the choices."""
    if os.path.exists(WEIGHTS):
        gpu_lib.selector_load(WEIGHTS)
    else:
        gpu_lib.selector_set_params(init_params(7))
    for A in (inputs.uniform(600, 600, seed=21), inputs.mixed_range(600, 64, (0, 8, 16), seed=22)):
        n = A.shape[0]
        b = inputs.vector(n, seed=23)
        dA = ColMajor.from_numpy(A)
        ipiv, info, st = gpu_lib.dgetrf(dA, nb=64, slices=0, stats=True)
        db = ColMajor.from_numpy(b)
        gpu_lib.dgetrs(dA, ipiv, db)
        gpu_lib.sync_status()
        assert int(info.item()) == 0
        assert 3 <= st.slices_min <= st.slices_max <= 8
        assert residual.backward_error(A, db.numpy()[:, 0], b) < 16


def test_selector_gain_over_fixed_slices(gpu_lib):
    """What the trained network gains over the method without it (mixed
    dynamic ranges, block rows scaled with r in {0, 8, 16}, n = 8192): LU +
    solve with slices chosen per step by the network and checked by the probe,
    against the constant s = 7 of the method and the fixed s = 8 fallback.
    Measured and asserted: every run passes the bar of 16; the network keeps
    the mean slice count near 7 (never below the 7 the data needs); against the
    constant s = 7 it gains nothing: it picks s = 7 on nearly every step and
    pays for the features, the probe and one host read of its prediction per
    step, so it is slower, by at most 2x at this size (the step count, not the
    work, sets that overhead)."""
    import torch
    gpu_lib.selector_load(WEIGHTS)
    n, nb = 8192, 256
    A = inputs.mixed_range(n, nb, (0, 8, 16), seed=8101)
    b = inputs.vector(n, seed=8102)
    A0 = ColMajor.from_numpy(A)
    b0 = ColMajor.from_numpy(b)
    res = {}
    for label, s in (("s7", 7), ("s8", 8), ("learned", 0)):
        W = ColMajor(A0.store.clone(), n, n)
        x = ColMajor(b0.store.clone(), n, 1)
        times = []
        for rep in range(3):
            W.store.copy_(A0.store)
            x.store.copy_(b0.store)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ipiv, info, st = gpu_lib.dgetrf(W, nb=nb, slices=s, stats=True)
            gpu_lib.dgetrs(W, ipiv, x)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        gpu_lib.sync_status()
        assert int(info.item()) == 0
        berr = residual.backward_error(A, x.numpy()[:, 0], b)
        res[label] = {"ms": min(times[1:]), "berr": berr, "mean_s": st.slices_mean, "failed": st.checks_failed}
    print(res)
    for v in res.values():
        assert v["berr"] < 16, res
    assert 7.0 <= res["learned"]["mean_s"] <= 7.5, res
    assert res["s7"]["ms"] < res["learned"]["ms"] < 2.0 * res["s7"]["ms"], res
