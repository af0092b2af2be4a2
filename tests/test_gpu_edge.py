"""Degenerate and edge cases of the CUDA path against the oracle (GPU)."""
import numpy as np
import pytest

from oracle import lb
from paper_1010_1233_gb300 import Sim, workloads as W
from paper_1010_1233_gb300 import _lib as L
from test_gpu_parity import FP32_TOL, FP64_TOL, _oracle, _rel

pytestmark = pytest.mark.gpu


def _fp64_parity(p, steps, f0=None):
    sim = Sim(p, precision="fp64")
    ref = _oracle(p)
    if f0 is not None:
        sim.set_populations(f0)
        ref.f = f0.copy()
    feq = lb.uniform_state(ref.p)
    scale = ref.f - feq                       # the initial deviation sets the scale (it may decay)
    worst = 0.0
    for _ in range(steps):
        sim.run(1)
        ref.run(1)
        worst = max(worst, _rel(sim.populations(), ref.f, scale))
    return worst, sim, ref


def test_zero_temperature_is_deterministic_relaxation():
    p = W.replica("D2Q9", 16, 8, W.taus_d2q9(0.7, 0.9, 1.3), kT=0.0, u0=(0.05, -0.02), seed=1)
    f0 = lb.uniform_state(lb.Params(**p)) * (1 + W.random_perturbation((9, 8, 16), 3, 1e-3))
    worst, sim, ref = _fp64_parity(p, 30, f0)
    assert worst < FP64_TOL
    again = Sim(p, precision="fp64")
    again.set_populations(f0)
    again.run(30)
    assert np.array_equal(again.populations(), sim.populations())          # no noise, no randomness


@pytest.mark.parametrize("nx,ny", [(2, 1), (2, 2), (4, 1)])
def test_smallest_lattices(nx, ny):
    p = W.replica("D2Q9", nx, ny, W.taus_d2q9(0.8), kT=1e-3, u0=(0.1, 0.0), seed=2, init_mode=1)
    worst, _, _ = _fp64_parity(p, 20)
    assert worst < FP64_TOL
    for vec in (1, 2):
        sim = Sim(p, precision="fp32")
        sim.set_step_config(vec, 0, 0)
        ref = _oracle(p)
        sim.run(10)
        ref.run(10)
        assert _rel(sim.populations(), ref.f, ref.f - lb.uniform_state(ref.p)) < FP32_TOL
    if nx % 4:
        with pytest.raises(L.FlbError):                                    # staged tiles need nx % 4 == 0
            Sim(p, precision="fp32").set_step_config(1, 0, 1)


def test_relaxation_time_near_one_half():
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.5005, 0.5005, 0.5005), kT=1e-4, seed=3, init_mode=1)
    worst, sim, _ = _fp64_parity(p, 50)
    assert worst < FP64_TOL
    assert np.all(np.isfinite(sim.conserved()))


def test_single_row_d2q9_with_sampling():
    p = W.replica("D2Q9", 32, 1, W.taus_d2q9(0.8), kT=1e-4, u0=(0.05, 0.0), seed=4, init_mode=1,
                  fields=(0, 9, 10))
    sim = Sim(p, precision="fp64")
    ref = _oracle(p)
    sim.run(30, 3)
    ref.run(30, 3)
    for a, b in [(0, 0), (0, 9), (9, 10)]:
        o = ref.acc.correlator(a, b)
        assert np.abs(sim.correlator(0, a, b) - o).max() < 1e-10 * max(1.0, np.abs(o).max())


def test_many_small_replicas_in_one_launch():
    reps = [W.replica("D2Q9", 8 * (1 + r % 3), 8, W.taus_d2q9(0.6 + 0.01 * r), kT=1e-4, u0=(0.005 * r, 0.0),
                      seed=r, stream=r, init_mode=1) for r in range(40)]
    sim = Sim(reps, precision="fp64")
    sim.run(15)
    for r in (0, 13, 27, 39):
        ref = _oracle(reps[r])
        ref.run(15)
        assert _rel(sim.populations(r), ref.f, ref.f - lb.uniform_state(ref.p)) < FP64_TOL
