"""Correlated noise for a moving fluid (noise_mode 1) on the CUDA path (GPU).

The library computes the noise root R on the host (Jacobi eigen-decomposition,
positive part, principal square root) and the kernels draw xi = s (R N); the
oracle computes R with numpy.  Parity against the FP64 oracle step by step, in
every step-kernel configuration, and the measured spectra against the linear
theory of the correlated scheme.
"""
import numpy as np
import pytest

from oracle import lb, mlp as omlp
from paper_1010_1233_gb300 import Sim, workloads as W
from test_gpu_parity import FP32_TOL, FP64_TOL, _oracle, _rel
from test_gpu_stats import compare, measure

pytestmark = pytest.mark.gpu

LADD = (1 << 3) | (1 << 4) | (1 << 5)
CASES = [
    ("D2Q9", 32, 16, dict(tau=W.taus_d2q9(0.8, 0.7, 1.1), u0=(0.2, 0.05))),
    ("D2Q9", 24, 10, dict(tau=W.taus_d2q9(0.6, 0.6, 1.0), u0=(-0.1, 0.15), noise_mask=LADD)),
    ("D2Q9", 16, 16, dict(tau=W.taus_d2q9(0.55, 0.55, 1.5), u0=(0.3, 0.1))),     # indefinite: positive part
    ("D1Q3", 64, 1, dict(tau=W.taus_d1q3(0.7), u0=(0.2, 0.0))),
]


@pytest.mark.parametrize("lat,nx,ny,kw", CASES, ids=[f"{c[0]}-{c[1]}x{c[2]}-{i}" for i, c in enumerate(CASES)])
def test_fp64_correlated_matches_oracle_every_step(lat, nx, ny, kw):
    p = W.replica(lat, nx, ny, kT=1e-3, seed=21, stream=2, init_mode=1, noise_mode=1, **kw)
    sim = Sim(p, precision="fp64")
    ref = _oracle(p)
    feq = lb.uniform_state(ref.p)
    worst = 0.0
    for _ in range(60):
        sim.run(1)
        ref.run(1)
        worst = max(worst, _rel(sim.populations(), ref.f, ref.f - feq))
    assert worst < FP64_TOL, worst
    # the correlated scheme really differs from the independent one at u0 != 0
    plain = _oracle(dict(p, noise_mode=0))
    plain.run(60)
    assert _rel(plain.f, ref.f, ref.f - feq) > 1e-3


@pytest.mark.parametrize("vec,staged,with_mlp", [(4, 0, False), (1, 0, False), (2, 1, False), (2, 0, True),
                                                 (1, 1, True)])
def test_fp32_correlated_every_kernel(vec, staged, with_mlp):
    p = W.replica("D2Q9", 64, 32, W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, u0=(0.15, -0.05), seed=4,
                  init_mode=1, noise_mode=1)
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


def test_correlated_spectra_match_theory():
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, u0=(0.15, 0.0), seed=17, init_mode=1,
                  fields=(0, W.FIELD_UX, W.FIELD_UY), noise_mode=1)
    meas = measure(p, "fp32", 20, 20000, 3000)
    zmax, dmax, S, ex = compare(p, meas)
    print(f"correlated u0 = 0.15: max |S - theory| = {dmax:.4f}, max z = {zmax:.2f}")
    assert zmax < 5.0
