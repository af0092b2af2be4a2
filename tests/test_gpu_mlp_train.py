"""Training kernels of the noise-scale network against the FP64 oracle (GPU)."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_1010_1233_gb300 import learned, workloads as W

pytestmark = pytest.mark.gpu


def _setup(R=3, B=300, K=40, seed=4):
    w = W.mlp_weights(seed, out_scale=0.3)
    X = np.stack([W.mlp_inputs(B, 10 + r) for r in range(R)]).astype(np.float32)
    Sp, G = W.correlator_tables(R, K, seed + 1)
    return w, X, Sp, G


def test_gradient_matches_oracle():
    w, X, Sp, G = _setup()
    tr = learned.Trainer(X, learned.gram(Sp, G), Sp.shape[2], w)
    loss, m, grad = tr.loss_and_grad()
    w64 = {k: v.astype(np.float64) for k, v in w.items()}
    L0, g0, _ = omlp.loss_grad(w64, X.astype(np.float64), Sp, G)
    _, m0 = omlp.loss(w64, X.astype(np.float64), Sp, G)
    assert abs(loss - L0) < 1e-5 * abs(L0)
    assert np.abs(m - m0).max() < 1e-5
    for k in w:
        scale = np.abs(g0[k]).max()
        assert np.abs(grad[k] - g0[k]).max() < 1e-4 * scale + 1e-9, k


def test_adam_step_matches_oracle():
    w, X, Sp, G = _setup(R=2, B=128, K=16, seed=7)
    tr = learned.Trainer(X, learned.gram(Sp, G), Sp.shape[2], w, lr=1e-2)
    # the Adam kernel against the published update applied to the kernel's own gradient
    # (near-zero gradients have no stable sign between FP32 and FP64, and Adam divides by |g|)
    w64 = {k: v.astype(np.float64) for k, v in w.items()}
    state = {}
    for _ in range(3):
        _, _, g = tr.loss_and_grad()
        w64 = omlp.adam_step(w64, {k: v.astype(np.float64) for k, v in g.items()}, state, lr=1e-2)
        tr.step()
        got = tr.weights()
        for k in w:
            assert np.abs(got[k] - w64[k]).max() < 1e-5 * max(1.0, np.abs(w64[k]).max()), k


def test_training_finds_exact_scales():
    # tables built so that constant scales s_c^2 = m*_c make the prediction exact:
    # S^plain = delta + sum_c (1 - m*_c) G^c; the trained network must approach m*
    w, X, _, G = _setup(R=4, B=256, K=64, seed=9)
    mstar = np.array([0.7, 1.2, 0.9, 1.3, 0.8, 1.1])
    T = omlp.targets(6)[None, :, None]
    Sp = T + np.einsum("c,rcpk->rpk", 1.0 - mstar, G)
    w["W3"] *= 0.1
    tr = learned.Trainer(X, learned.gram(Sp, G), Sp.shape[2], w, lr=3e-3)
    l0 = tr.loss_and_grad()[0]
    tr.step(1500)
    l1, m, _ = tr.loss_and_grad()
    print(f"loss {l0:.3g} -> {l1:.3g}; m = {np.round(m.mean(0), 3)}")
    assert l1 < 0.05 * l0
    assert np.abs(m.mean(0) - mstar).max() < 0.05
