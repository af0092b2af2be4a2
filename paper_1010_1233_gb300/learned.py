"""Learned noise-scale correction: training data from the plain method, GPU training, evaluation.

Sec. 3 of the paper reports that at large mean velocity the moment fluctuations
stop decoupling (Galilean-invariance violation).  The learned extension (not
in the paper) rescales the Eq. 8 noise amplitude of each non-conserved D2Q9
moment by s_c(u_x, u_y, rho - rho0) from a 3-32-32-6 network.  It is trained on
what the plain method itself measures:

* for every training mean velocity u0 the plain run gives S^plain_p(k) of the six
  hydrodynamic pairs, and six runs with only the noise of moment 3 + c on give
  the response G^c_p(k) (the equal-time covariance is linear in the noise
  variances, so S(s) = S^plain + sum_c (<s_c^2> - 1) G^c);
* per-site inputs (u_x, u_y, rho - rho0) are taken from the plain run's sampled fields;
* the loss is the mean of |S(s) - delta_p|^2 over runs, included k and pairs
  (the Galilean-invariant ideal gas: S_rho_rho = S_uxux = S_uyuy = 1, cross pairs 0).

All arithmetic runs in libflb kernels (flb_mlp_gram, flb_mlp_train_step);
this module marshals arrays and sequences the calls.
"""
import ctypes

import numpy as np
import torch

from . import _lib as L
from .sim import Sim
from . import workloads as W

HYDRO_FIELDS = (0, W.FIELD_UX, W.FIELD_UY)
HYDRO_PAIRS = ((0, 0), (0, 9), (0, 10), (9, 9), (9, 10), (10, 10))
NONCONSERVED = (3, 4, 5, 6, 7, 8)
N_PARAMS = 32 * 3 + 32 * 32 + 6 * 32 + 32 + 32 + 6


def pack(w):
    return np.concatenate([np.asarray(w[k], np.float32).ravel() for k in ("W1", "W2", "W3", "b1", "b2", "b3")])


def unpack(v):
    v = np.asarray(v, np.float32)
    out, off = {}, 0
    for k, shape in (("W1", (32, 3)), ("W2", (32, 32)), ("W3", (6, 32)), ("b1", (32,)), ("b2", (32,)), ("b3", (6,))):
        n = int(np.prod(shape))
        out[k] = v[off:off + n].reshape(shape).copy()
        off += n
    return out


def included_k(nx, ny):
    """Mask of wave vectors compared with theory: k = 0 (conserved) and the neutral
    modes (pi, 0), (0, pi), where a momentum component only flips sign, are excluded."""
    m = np.ones((ny, nx), bool)
    m[0, 0] = False
    m[0, nx // 2] = False
    m[ny // 2, 0] = False
    return m


def gram(Splain, G, stream=None):
    """(d0, g, H) per run on the device from S^plain (R, 6, K) and G (R, 6, 6, K), complex."""
    R, P, K = Splain.shape
    sp = torch.tensor(np.stack([Splain.real, Splain.imag], -1), dtype=torch.float64, device="cuda").contiguous()
    g = torch.tensor(np.stack([G.real, G.imag], -1), dtype=torch.float64, device="cuda").contiguous()
    out = torch.empty((R, 43), dtype=torch.float64, device="cuda")
    st = stream or torch.cuda.current_stream()
    L.check(L.lib().flb_mlp_gram(ctypes.c_void_p(sp.data_ptr()), ctypes.c_void_p(g.data_ptr()), R, P, K,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream)))
    return out


class Trainer:
    """Adam on the network weights with the correlator loss (GPU kernels)."""

    def __init__(self, X, gram_dev, K, weights, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        X = np.asarray(X, np.float32)
        self.R, self.B = X.shape[0], X.shape[1]
        self.K = int(K)
        self.X = torch.tensor(X, device="cuda").contiguous()
        self.gram = gram_dev
        self.w = torch.tensor(pack(weights), device="cuda")
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.t = 0
        self.lr, self.betas, self.eps = lr, betas, eps
        nb = ctypes.c_size_t()
        L.check(L.lib().flb_mlp_scratch_bytes(self.R, self.B, ctypes.byref(nb)))
        self.scratch = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.msq = torch.zeros((self.R, 6), dtype=torch.float64, device="cuda")
        self.grad = torch.zeros_like(self.w)

    def _call(self, lr):
        st = torch.cuda.current_stream()
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        L.check(L.lib().flb_mlp_train_step(p(self.w), p(self.m), p(self.v), self.t, float(lr), self.betas[0],
                                           self.betas[1], self.eps, p(self.X), self.R, self.B, p(self.gram), 6,
                                           self.K, p(self.loss), p(self.msq), p(self.grad), p(self.scratch),
                                           self.scratch.numel(), ctypes.c_void_p(st.cuda_stream)))

    def loss_and_grad(self):
        """Loss, <s^2> per run and channel, gradient at the current weights (no update)."""
        self._call(0.0)
        torch.cuda.synchronize()
        return float(self.loss.item()), self.msq.cpu().numpy(), unpack(self.grad.cpu().numpy())

    def step(self, n=1):
        for _ in range(n):
            self.t += 1
            self._call(self.lr)
        return self

    def weights(self):
        return unpack(self.w.cpu().numpy())


def run_spectra(replicas, steps, warmup, sample_every, precision="fp32", mlp=None):
    """Batched run; returns the Sim (correlators accumulated after the warm-up)."""
    sim = Sim(replicas, precision=precision)
    if mlp is not None:
        sim.set_mlp(mlp)
    sim.run(warmup)
    sim.reset_stats()
    sim.run(steps, sample_every)
    return sim


def hydro_matrix(sim, r, mask):
    """The six hydrodynamic correlators of replica r at the included k, (6, K) complex."""
    return np.stack([sim.correlator(r, a, b)[mask] for a, b in HYDRO_PAIRS])


def collect(u0s, n=128, tau=(0.8, 0.8, 1.0), kT=1e-4, steps=100_000, warmup=10_000, sample_every=10,
            n_inputs=4096, seed=100):
    """Plain and single-channel runs at each training u0; returns S^plain, G, inputs X, K."""
    reps = []
    for i, u in enumerate(u0s):
        for ch in (None,) + NONCONSERVED:
            mask = None if ch is None else (1 << ch)
            reps.append(W.replica("D2Q9", n, n, W.taus_d2q9(*tau), kT=kT, u0=(u, 0.0), seed=seed + 7 * i,
                                  stream=len(reps), noise_mask=mask, init_mode=1, fields=HYDRO_FIELDS))
    sim = run_spectra(reps, steps, warmup, sample_every)
    km = included_k(n, n)
    R = len(u0s)
    Sp = np.zeros((R, 6, km.sum()), complex)
    G = np.zeros((R, 6, 6, km.sum()), complex)
    X = np.zeros((R, n_inputs, 3), np.float32)
    rng = np.random.default_rng(seed)
    for i, u in enumerate(u0s):
        base = 7 * i
        Sp[i] = hydro_matrix(sim, base, km)
        for c in range(6):
            G[i, c] = hydro_matrix(sim, base + 1 + c, km)
        f = sim.fields(base)                                   # last sample, [field][ny][nx]
        idx = rng.choice(n * n, n_inputs, replace=False)
        X[i, :, 0] = f[1].ravel()[idx] + u                     # u_x
        X[i, :, 1] = f[2].ravel()[idx]                         # u_y
        X[i, :, 2] = f[0].ravel()[idx]                         # rho - rho0
    sim.close()
    return dict(Splain=Sp, G=G, X=X, K=int(km.sum()), u0s=list(u0s), n=n)


def error_metrics(S6, target=None):
    """max and RMS of |S - delta| over the six pairs and included k."""
    t = np.array([1, 0, 0, 1, 0, 1], float)[:, None] if target is None else target
    d = np.abs(S6 - t)
    return float(d.max()), float(np.sqrt(np.mean(d**2)))


def experiment(n=128, n_train=16, u_max=0.3, heldout=(0.07, 0.17, 0.2, 0.27), steps=100_000, warmup=10_000,
               sample_every=10, iters=2000, lr=3e-3, seed=0):
    """The learned-correction workload: train on plain-method data, evaluate held out."""
    import time
    t0 = time.time()
    u0s = [u_max * i / (n_train - 1) for i in range(n_train)]
    data = collect(u0s, n=n, steps=steps, warmup=warmup, sample_every=sample_every)
    t1 = time.time()
    tr = Trainer(data["X"], gram(data["Splain"], data["G"]), data["K"], W.mlp_weights(seed, out_scale=0.01), lr=lr)
    l0 = tr.loss_and_grad()[0]
    tr.step(iters)
    l1, msq, _ = tr.loss_and_grad()
    t2 = time.time()
    w = tr.weights()
    out = dict(n=n, train_u0=u0s, loss_before=l0, loss_after=l1, collect_s=t1 - t0, train_s=t2 - t1,
               mean_s2=msq.tolist(), heldout={})
    km = included_k(n, n)
    for u in heldout:
        res = {}
        # the plain method, the learned per-site scales, and (for comparison) the correlated
        # noise of the moving equilibrium (noise_mode 1), which needs no training
        for name, mlp, mode in (("plain", None, 0), ("learned", w, 0), ("correlated", None, 1)):
            p = W.replica("D2Q9", n, n, W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, u0=(u, 0.0), seed=999,
                          init_mode=1, fields=HYDRO_FIELDS, noise_mode=mode)
            sim = run_spectra([p], steps, warmup, sample_every, mlp=mlp)
            S = hydro_matrix(sim, 0, km)
            sim.close()
            mx, rms = error_metrics(S)
            res[name] = dict(max_err=mx, rms_err=rms)
        out["heldout"][str(u)] = res
    return out, w


if __name__ == "__main__":
    import json
    import sys
    quick = "--quick" in sys.argv
    kw = dict(n=32, n_train=4, steps=20_000, warmup=2_000, sample_every=5, iters=600) if quick else {}
    res, _ = experiment(**kw)
    print(json.dumps(res))
