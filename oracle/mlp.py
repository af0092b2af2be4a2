"""Per-site noise-scale network and its correlator loss, FP64 (test infrastructure only).

This is a learned extension, not part of the paper.  Sec. 3 reports that at a
large mean velocity the moment fluctuations no longer decouple (Eq. 7 needs
u << 1), i.e. Galilean invariance is violated.  The extension rescales the
Eq. 8 noise amplitude of each non-conserved D2Q9 moment a = 3..8 per site:
xi^a -> s_a xi^a with s = 1 + o(x) and

    x  = (u_x, u_y, rho - rho0)
    h1 = relu(W1 x + b1)     W1: 32 x 3
    h2 = relu(W2 h1 + b2)    W2: 32 x 32
    o  = W3 h2 + b3          W3: 6 x 32

Loss.  For training runs r at mean velocities u0_r the plain method gives
measured normalised correlators S^plain_{r,p}(k) of the six hydrodynamic pairs
p in {rho rho, rho u_x, rho u_y, u_x u_x, u_x u_y, u_y u_y}, and runs with the
noise of only channel c switched on give its response G^c_{r,p}(k).  The
equal-time covariance is linear in the noise variances, so with scales s the
prediction is

    S_{r,p}(k) = S^plain_{r,p}(k) + sum_c (m_{r,c} - 1) G^c_{r,p}(k),
    m_{r,c} = mean over the run's sampled sites b of s_c(x_{r,b})^2,

and the loss is the mean of |S_{r,p}(k) - delta_p|^2 over runs, included k and
pairs (delta_p = 1 for the three autocorrelations, 0 for the cross pairs; the
Galilean-invariant ideal gas).

Parity: forward pinned by special cases (zero output layer gives s = 1, a
single-unit network equals its closed form); backward pinned by central finite
differences of the loss; Adam (Kingma & Ba, 2015) by the closed form of its first
two steps on a gradient that flips sign (state carried, bias correction at t = 2)
and against an installed independent implementation (torch.optim.Adam, FP64)
over 40 steps.
"""
import numpy as np

HIDDEN = 32
N_IN = 3
N_OUT = 6
AUTO_PAIRS = (0, 3, 5)      # index of rho-rho, ux-ux, uy-uy in the six hydrodynamic pairs


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even), via float32, as FP64 values."""
    f = np.asarray(x, dtype=np.float32).copy()
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(w, X, bf16_operands=False):
    """Forward pass on features X (B, 3); returns the intermediate arrays and s (B, 6).

    bf16_operands=True rounds the inputs, the biases and both hidden activations to
    bfloat16 before each matrix product, as a tensor-core inference kernel with
    bfloat16 operands (the bias as the weight of a constant-1 input) and FP32
    accumulation does (weights are expected already rounded).
    """
    rnd = to_bf16 if bf16_operands else (lambda a: np.asarray(a, dtype=np.float64))
    X = rnd(X)
    z1 = X @ w["W1"].T + rnd(w["b1"])
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ w["W2"].T + rnd(w["b2"])
    h2 = rnd(np.maximum(z2, 0.0))
    o = h2 @ w["W3"].T + rnd(w["b3"])
    return dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, o=o, s=1.0 + o)


def predicted_correlators(m, Splain, G):
    """S_{r,p}(k) = S^plain + sum_c (m_{r,c} - 1) G^c.  Splain (R, P, K), G (R, C, P, K)."""
    return Splain + np.einsum("rc,rcpk->rpk", m - 1.0, G)


def targets(P):
    t = np.zeros(P)
    t[list(AUTO_PAIRS)] = 1.0
    return t


def loss(w, Xruns, Splain, G):
    """Loss of the module docstring; Xruns (R, B, 3), Splain (R, P, K), G (R, C, P, K)."""
    R = Xruns.shape[0]
    m = np.stack([np.mean(forward(w, Xruns[r])["s"] ** 2, axis=0) for r in range(R)])
    S = predicted_correlators(m, Splain, G)
    T = targets(S.shape[1])[None, :, None]
    return float(np.mean(np.abs(S - T) ** 2)), m


def loss_grad(w, Xruns, Splain, G):
    """Analytic gradient of ``loss`` with respect to every weight and bias."""
    R, B, _ = Xruns.shape
    P, K = Splain.shape[1], Splain.shape[2]
    L, m = loss(w, Xruns, Splain, G)
    S = predicted_correlators(m, Splain, G)
    T = targets(P)[None, :, None]
    scale = 2.0 / (R * P * K)
    dm = scale * np.einsum("rpk,rcpk->rc", np.conj(S - T), G).real      # dL/dm_{r,c}
    grads = {k: np.zeros_like(v) for k, v in w.items()}
    for r in range(R):
        fw = forward(w, Xruns[r])
        do = dm[r][None, :] * 2.0 * fw["s"] / B                          # dL/do (B, 6)
        grads["W3"] += do.T @ fw["h2"]
        grads["b3"] += do.sum(axis=0)
        dz2 = (do @ w["W3"]) * (fw["z2"] > 0)
        grads["W2"] += dz2.T @ fw["h1"]
        grads["b2"] += dz2.sum(axis=0)
        dz1 = (dz2 @ w["W2"]) * (fw["z1"] > 0)
        grads["W1"] += dz1.T @ fw["X"]
        grads["b1"] += dz1.sum(axis=0)
    return L, grads, dm


def adam_step(w, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, 2015) with bias correction; state holds m, v, t."""
    t = state.get("t", 0) + 1
    out = {}
    for k in w:
        m = beta1 * state.get(("m", k), 0.0) + (1.0 - beta1) * g[k]
        v = beta2 * state.get(("v", k), 0.0) + (1.0 - beta2) * g[k] ** 2
        state[("m", k)], state[("v", k)] = m, v
        mhat = m / (1.0 - beta1**t)
        vhat = v / (1.0 - beta2**t)
        out[k] = w[k] - lr * mhat / (np.sqrt(vhat) + eps)
    state["t"] = t
    return out
