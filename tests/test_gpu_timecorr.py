"""Time correlators F_ab(k, tau) at selected wave vectors on the CUDA path (GPU).

The column pass of every sample writes X_f(k_j) of the selected wave vectors to a
ring of the last n_lags samples; a small kernel adds X_a(k, s) X_b(k, s - tau)^*.
Parity with the oracle's TimeAccumulator on the same run (ring wrapped, batched
replicas, graphs on and off), and the measured values against the linear theory.
"""
import numpy as np
import pytest

from oracle import lb, spectra, theory
from paper_1010_1233_gb300 import Sim, workloads as W
from paper_1010_1233_gb300 import _lib as L

pytestmark = pytest.mark.gpu

KS = [(0, 1), (1, 0), (2, 3), (8, 5), (15, 8)]          # (ky, kx): includes kx = nx/2 and ky > ny/2


def _oracle_run(p, ks, T, steps, every):
    r = lb.Run(lb.Params(**p), time_k=ks, n_lags=T)
    r.run(steps, every)
    return r


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_time_correlators_match_oracle(precision, tol):
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8, 0.7, 1.0), kT=1e-4, u0=(0.1, 0.05), seed=5, init_mode=1,
                  fields=(0, 9, 10))
    T = 5
    sim = Sim(p, precision=precision)
    sim.set_time_correlator(KS, T)
    sim.run(40, 3)                                   # 14 samples: the ring of 5 wraps
    ref = _oracle_run(p, KS, T, 40, 3)
    for a in p["fields"]:
        for b in p["fields"]:
            g, n = sim.time_correlator(0, a, b, with_count=True)
            o = ref.tacc.correlator(a, b)
            assert n == ref.tacc.n == 14
            assert np.abs(g - o).max() < tol * max(1.0, np.abs(o).max()), (a, b)


def test_batched_replicas_and_graphs():
    reps = [W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8), kT=1e-4, u0=(0.05, 0.0), seed=1, stream=1, init_mode=1,
                      fields=(0, 9)),
            W.replica("D2Q9", 32, 16, W.taus_d2q9(0.7), kT=1e-4, u0=(0.0, 0.1), seed=2, stream=2, init_mode=1,
                      fields=(0, 9, 10))]
    T, steps, every = 4, 80, 2                      # 80 steps: two graph chunks of 32 steps and direct steps
    outs = []
    for graphs in (True, False):
        sim = Sim(reps, precision="fp32")
        sim.set_graphs(graphs)
        sim.set_time_correlator(KS, T)
        sim.run(steps, every)
        outs.append([sim.time_correlator(r, 0, 9) for r in range(2)])
    for r in range(2):
        assert np.array_equal(outs[0][r], outs[1][r])              # graph replay changes nothing
        ref = _oracle_run(reps[r], KS, T, steps, every)
        o = ref.tacc.correlator(0, 9)
        assert np.abs(outs[0][r] - o).max() < 2e-4 * max(1.0, np.abs(o).max())


def test_reset_off_and_errors():
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8), kT=1e-4, seed=3, fields=(0,))
    sim = Sim(p, precision="fp32")
    sim.set_time_correlator([(0, 1)], 3)
    sim.run(10, 1)
    v, n = sim.time_correlator(0, 0, 0, with_count=True)
    assert n == 10 and np.all(np.isfinite(v))
    sim.reset_stats()
    v, n = sim.time_correlator(0, 0, 0, with_count=True)
    assert n == 0 and np.all(np.isnan(v))
    for bad in ([(0, 0)], [(0, 9)], [(16, 1)]):                     # k = 0, kx > nx/2, ky >= ny
        with pytest.raises(L.FlbError):
            sim.set_time_correlator(bad, 3)
    sim.set_time_correlator([], 0)
    sim.run(5, 1)                                                   # off: sampling goes on without them


def test_time_correlators_match_theory():
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, u0=(0.1, 0.0), seed=9, init_mode=1,
                  fields=(0, 9))
    ks, T, every = [(0, 1), (1, 2), (3, 0), (0, 6)], 6, 2
    F = theory.time_correlators(lb.Params(**p), list(p["fields"]), ks, T, every)
    sim = Sim(p, precision="fp32")
    sim.set_time_correlator(ks, T)
    sim.run(2000)
    batches = {pr: [] for pr in F}
    for _ in range(20):
        sim.reset_stats()
        sim.run(20000, every)
        for pr in batches:
            batches[pr].append(sim.time_correlator(0, *pr))
    worst = 0.0
    for pr, v in batches.items():
        m = np.mean(v, 0)
        se = np.std(v, 0, ddof=1) / np.sqrt(len(v))
        for part in (np.real, np.imag):
            worst = max(worst, (np.abs(part(m) - part(F[pr])) / np.maximum(se, 2e-3)).max())
    print(f"time correlators vs theory: max z = {worst:.2f}")
    assert worst < 5.0


def test_kernel_launch_count_with_time_correlators():
    # flb_kernel_launches with time correlators, which take every sample on its own: per
    # sample the row transform, the column pass with the pair sums and the ring entries,
    # the lagged products and the ring advance (D2Q9); the direct transforms at the wave
    # vectors, their finishing pass, the lagged products and the ring advance (D3Q15)
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8), kT=1e-4, seed=3, init_mode=1, fields=(0, W.FIELD_UX))
    sim = Sim(p, precision="fp32")
    sim.set_graphs(False)
    sim.set_time_correlator([(1, 2), (3, 0)], 2)
    n0 = sim.kernel_launches()
    sim.run(3, 1)
    assert sim.kernel_launches() - n0 == 3 + 3 * (1 + 1 + 2)
    sim.close()
    q = W.replica3(8, 6, 4, W.taus_d3q15(0.8), kT=1e-4, seed=3, init_mode=1, fields=(0, 4))
    sim = Sim(q, precision="fp32")
    sim.set_graphs(False)
    sim.set_time_correlator([(0, 0, 1), (1, 2, 3)], 2)
    n0 = sim.kernel_launches()
    sim.run(3, 1)
    assert sim.kernel_launches() - n0 == 3 + 3 * 4
    sim.close()
