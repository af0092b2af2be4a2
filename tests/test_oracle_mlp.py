"""Pins of the oracle's noise-scale network, its loss gradient and Adam (CPU only)."""
import numpy as np
import pytest

from oracle import mlp
from paper_1010_1233_gb300 import workloads as W


def _w64(seed, **kw):
    return {k: v.astype(np.float64) for k, v in W.mlp_weights(seed, **kw).items()}


def test_zero_output_layer_is_plain_method():
    w = _w64(0)
    w["W3"][:] = 0
    w["b3"][:] = 0
    s = mlp.forward(w, W.mlp_inputs(100, 1))["s"]
    assert np.all(s == 1.0)


def test_single_unit_closed_form():
    # hidden width 1 (others zeroed): s_c = 1 + b3_c + W3_c relu(W2 relu(W1 x + b1) + b2)
    w = _w64(2)
    for k in ("W1", "b1"):
        w[k][1:] = 0
    w["W2"][:] = 0
    w["W2"][0, 0] = 0.7
    w["b2"][:] = 0
    w["b2"][0] = -0.05
    w["W3"][:, 1:] = 0
    X = W.mlp_inputs(50, 3)
    h = np.maximum(X @ w["W1"][0] + w["b1"][0], 0)
    h2 = np.maximum(0.7 * h - 0.05, 0)
    want = 1 + w["b3"][None, :] + h2[:, None] * w["W3"][:, 0][None, :]
    assert np.abs(mlp.forward(w, X)["s"] - want).max() < 1e-14


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -0.1, 3.0e-3])
    r = mlp.to_bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2**-6   # ties to even
    assert np.all(np.abs(r - x) <= np.abs(x) * 2**-8)


def test_loss_gradient_matches_finite_differences():
    w = _w64(4)
    R, B, K = 3, 64, 20
    X = np.stack([W.mlp_inputs(B, 10 + r) for r in range(R)])
    Sp, G = W.correlator_tables(R, K, 5)
    L0, g, _ = mlp.loss_grad(w, X, Sp, G)
    rng = np.random.default_rng(0)
    for k in w:
        for _ in range(4):
            idx = tuple(rng.integers(0, n) for n in w[k].shape)
            h = 1e-6
            wp = {kk: vv.copy() for kk, vv in w.items()}
            wm = {kk: vv.copy() for kk, vv in w.items()}
            wp[k][idx] += h
            wm[k][idx] -= h
            fd = (mlp.loss(wp, X, Sp, G)[0] - mlp.loss(wm, X, Sp, G)[0]) / (2 * h)
            assert abs(fd - g[k][idx]) < 1e-6 * max(1.0, abs(fd)), (k, idx, fd, g[k][idx])


def test_loss_zero_when_prediction_exact():
    # if S^plain = delta and the network gives s = 1, the loss vanishes
    w = _w64(6)
    w["W3"][:] = 0
    w["b3"][:] = 0
    R, K = 2, 7
    Sp = np.broadcast_to(mlp.targets(6)[None, :, None], (R, 6, K)).astype(complex)
    G = W.correlator_tables(R, K, 7)[1]
    L, m = mlp.loss(w, np.stack([W.mlp_inputs(8, r) for r in range(R)]), Sp, G)
    assert L == 0.0 and np.all(m == 1.0)


def test_adam_first_step_is_signed_lr():
    # bias-corrected first Adam step moves each weight by lr * g / (|g| + eps)
    w = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -1e-3, 2.0])}
    out = mlp.adam_step(w, g, {}, lr=0.01, eps=1e-8)
    assert np.allclose(out["a"], w["a"] - 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8), rtol=0, atol=1e-15)


def test_adam_alternating_gradient_closed_form():
    # g, then -g: m2 = -(1 - b1)^2 g, v2 = (1 - b2^2) g^2, so the bias-corrected second step
    # is -lr (1 - b1) / (1 + b1) sign(g) (up to eps): state carried, t = 2 in the correction
    b1, b2, lr = 0.9, 0.999, 0.01
    w = {"a": np.array([1.0, -2.0, 0.5, 3.0])}
    g = np.array([0.3, -0.7, 2.0, 1e-2])
    st = {}
    w1 = mlp.adam_step(w, {"a": g}, st, lr=lr, beta1=b1, beta2=b2, eps=0.0)
    w2 = mlp.adam_step(w1, {"a": -g}, st, lr=lr, beta1=b1, beta2=b2, eps=0.0)
    assert st["t"] == 2
    assert np.allclose(w1["a"] - w["a"], -lr * np.sign(g), rtol=0, atol=1e-15)
    assert np.allclose(w2["a"] - w1["a"], lr * (1 - b1) / (1 + b1) * np.sign(g), rtol=0, atol=1e-15)


def test_adam_matches_torch_optimizer_over_many_steps():
    # an installed, independent Adam (torch.optim.Adam on the CPU, FP64) over 40 steps of
    # varying gradients on two parameter arrays
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    w = {"a": rng.normal(size=(5, 3)), "b": rng.normal(size=7)}
    params = {k: torch.tensor(v.copy(), dtype=torch.float64, requires_grad=True) for k, v in w.items()}
    opt = torch.optim.Adam(list(params.values()), lr=3e-3, betas=(0.8, 0.99), eps=1e-7)
    st = {}
    for _ in range(40):
        g = {k: rng.normal(size=v.shape) * rng.uniform(0.01, 3.0) for k, v in w.items()}
        w = mlp.adam_step(w, g, st, lr=3e-3, beta1=0.8, beta2=0.99, eps=1e-7)
        opt.zero_grad()
        for k, p in params.items():
            p.grad = torch.tensor(g[k], dtype=torch.float64)
        opt.step()
    for k, p in params.items():
        assert np.abs(w[k] - p.detach().numpy()).max() < 1e-12, k
