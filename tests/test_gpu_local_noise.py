"""Local-density noise amplitude (noise_mode 2) on the CUDA path (GPU)."""
import numpy as np
import pytest

from oracle import lb, mlp as omlp
from paper_1010_1233_gb300 import Sim, workloads as W
from test_gpu_parity import FP32_TOL, FP64_TOL, _oracle, _rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("lat,nx,ny,tau,u0", [("D2Q9", 32, 16, W.taus_d2q9(0.8, 0.7, 1.1), (0.1, 0.05)),
                                              ("D1Q3", 48, 1, W.taus_d1q3(0.7), (0.15, 0.0))])
def test_fp64_local_amplitude_matches_oracle(lat, nx, ny, tau, u0):
    p = W.replica(lat, nx, ny, tau, kT=1e-2, u0=u0, seed=8, init_mode=1, noise_mode=2)
    sim = Sim(p, precision="fp64")
    ref = _oracle(p)
    feq = lb.uniform_state(ref.p)
    worst = 0.0
    for _ in range(40):
        sim.run(1)
        ref.run(1)
        worst = max(worst, _rel(sim.populations(), ref.f, ref.f - feq))
    assert worst < FP64_TOL, worst
    glob = _oracle(dict(p, noise_mode=0))
    glob.run(40)
    assert _rel(glob.f, ref.f, ref.f - feq) > 1e-4          # the local factor is seen


@pytest.mark.parametrize("vec,staged,with_mlp", [(4, 0, False), (2, 1, False), (2, 0, True)])
def test_fp32_local_amplitude_every_kernel(vec, staged, with_mlp):
    p = W.replica("D2Q9", 64, 32, W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-3, u0=(0.1, 0.0), seed=6, init_mode=1,
                  noise_mode=2)
    sim = Sim(p, precision="fp32")
    ref = _oracle(p)
    tol = FP32_TOL
    if with_mlp:
        wts = W.mlp_weights(3, out_scale=0.5)
        sim.set_mlp(wts)
        ref.p.mlp = {k: (omlp.to_bf16(v) if k.startswith("W") else v.astype(np.float64)) for k, v in wts.items()}
        ref.p.mlp_bf16 = True
        tol = 1e-3
    sim.set_step_config(vec, 0, staged)
    sim.run(20)
    ref.run(20)
    assert _rel(sim.populations(), ref.f, ref.f - lb.uniform_state(ref.p)) < tol
