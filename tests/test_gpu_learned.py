"""The learned noise-scale correction, end to end on the GPU (small lattices).

Plain and single-channel runs at training mean velocities give the loss tables;
the network is trained by the library's kernels; at a held-out mean velocity
the corrected method must lie closer to the Galilean-invariant ideal gas than
the plain method, and its measured spectra must agree with the linear theory
evaluated at the network's average noise scales.
"""
import numpy as np
import pytest

from oracle import lb, theory
from paper_1010_1233_gb300 import learned, workloads as W

pytestmark = pytest.mark.gpu

N, TAU = 32, (0.8, 0.8, 1.0)


def _held_out(u0, mlp, seed):
    p = W.replica("D2Q9", N, N, W.taus_d2q9(*TAU), kT=1e-4, u0=(u0, 0.0), seed=seed, init_mode=1,
                  fields=learned.HYDRO_FIELDS)
    sim = learned.run_spectra([p], 40_000, 4_000, 5, mlp=mlp)
    km = learned.included_k(N, N)
    S = learned.hydro_matrix(sim, 0, km)
    X = sim.fields(0)
    sim.close()
    return p, S, km, X


def test_learned_correction_beats_plain_at_held_out_velocity():
    data = learned.collect((0.0, 0.1, 0.2, 0.3), n=N, tau=TAU, steps=30_000, warmup=3_000, sample_every=5,
                           n_inputs=1024)
    tr = learned.Trainer(data["X"], learned.gram(data["Splain"], data["G"]), data["K"],
                         W.mlp_weights(0, out_scale=0.01), lr=3e-3)
    l0 = tr.loss_and_grad()[0]
    tr.step(600)
    l1, msq, _ = tr.loss_and_grad()
    print(f"training loss {l0:.4g} -> {l1:.4g}; <s^2> at u0=0.3: {np.round(msq[-1], 3)}")
    assert l1 < l0
    w = tr.weights()
    u0 = 0.25
    p, S_plain, km, _ = _held_out(u0, None, 77)
    _, S_learn, _, X = _held_out(u0, w, 77)
    e_plain = learned.error_metrics(S_plain)
    e_learn = learned.error_metrics(S_learn)
    print(f"u0 = {u0}: plain max/rms {e_plain[0]:.3f}/{e_plain[1]:.4f}, "
          f"learned max/rms {e_learn[0]:.3f}/{e_learn[1]:.4f}")
    assert e_learn[1] < e_plain[1]
    # the corrected spectra follow the linear theory at the network's mean scales
    from oracle import mlp as omlp
    feats = np.stack([X[1].ravel() + u0, X[2].ravel(), X[0].ravel()], 1)
    w64 = {k: (omlp.to_bf16(v) if k.startswith("W") else v.astype(np.float64)) for k, v in w.items()}
    s = omlp.forward(w64, feats, bf16_operands=True)["s"]
    scale = np.sqrt(np.mean(s**2, axis=0))
    P = lb.Params(**p)
    St, ex = theory.theory_spectra(P, list(learned.HYDRO_FIELDS), scale=scale)
    pred = np.stack([St[pr][km] for pr in learned.HYDRO_PAIRS])
    dev = np.abs(S_learn - pred)
    print(f"learned vs theory at mean scales: max {dev.max():.3f}, rms {np.sqrt(np.mean(dev**2)):.4f}")
    assert np.sqrt(np.mean(dev**2)) < 0.6 * e_plain[1] + 0.02
