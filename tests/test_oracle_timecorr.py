"""Time correlators F_ab(k, tau) at selected wave vectors (oracle, CPU only).

An extension of the equal-time correlators of Eqs. 11-12 (the paper leaves the
dynamics to future work): F_ab(k, tau) = N^{ab} <X_a(k, s) X_b(k, s - tau)^*>.
The linear theory propagates the stationary covariance with the one-step
operator; the oracle's simulated values must agree within batch-means errors.
"""
import numpy as np
import pytest

from oracle import lb, spectra, theory
from paper_1010_1233_gb300 import workloads as W


def _params(**kw):
    return lb.Params(**W.replica(**kw))


def test_zero_lag_is_the_equal_time_correlator():
    p = _params(nx=8, ny=8, tau=W.taus_d2q9(0.8, 0.7, 1.0), kT=1e-4, seed=3, u0=(0.1, 0.0), init_mode=1,
                fields=[0, 9, 10])
    ks = [(0, 1), (3, 2), (5, 4)]
    r = lb.Run(p, time_k=ks, n_lags=4)
    r.run(60, 2)
    for a in p.fields:
        for b in p.fields:
            c = r.acc.correlator(a, b)
            want = np.array([c[ky, kx] for ky, kx in ks])
            assert np.abs(r.tacc.correlator(a, b)[0] - want).max() < 1e-12
    # theory: lag 0 is the equal-time prediction
    S, _ = theory.theory_spectra(p, p.fields)
    F = theory.time_correlators(p, p.fields, ks, 3, 2)
    for (a, b), v in S.items():
        assert np.abs(F[(a, b)][0] - np.array([v[ky, kx] for ky, kx in ks])).max() < 1e-12


@pytest.mark.parametrize("case", ["d1q3", "d2q9_moving"])
def test_simulated_time_correlators_match_theory(case):
    if case == "d1q3":
        p = _params(lattice="D1Q3", nx=16, ny=1, tau=W.taus_d1q3(0.8), kT=1e-4, seed=1, init_mode=1,
                    fields=[0, 1])
        ks, T, every, nb, steps, warm = [(0, 1), (0, 2), (0, 5)], 6, 1, 12, 1200, 0
    else:
        p = _params(nx=8, ny=8, tau=W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, seed=4, u0=(0.15, 0.0),
                    init_mode=1, fields=[0, 9])
        ks, T, every, nb, steps, warm = [(0, 1), (1, 2), (3, 0)], 5, 2, 10, 800, 300
    F = theory.time_correlators(p, p.fields, ks, T, every)
    r = lb.Run(p)
    r.run(warm)
    batches = {pr: [] for pr in F}
    for _ in range(nb):
        r.tacc = spectra.TimeAccumulator(p, ks, T)
        r.acc = spectra.Accumulator(p)
        r.run(steps, every)
        for pr in batches:
            batches[pr].append(r.tacc.correlator(*pr))
    worst = 0.0
    for pr, v in batches.items():
        m = np.mean(v, 0)
        se = np.std(v, 0, ddof=1) / np.sqrt(nb)
        for part in (np.real, np.imag):
            worst = max(worst, (np.abs(part(m) - part(F[pr])) / np.maximum(se, 1e-3)).max())
    assert worst < 5.0, worst


def test_conjugation_and_time_direction_matter():
    # a conjugation slip (X_a^* X_b) or a reversed lag (X_a(s - tau) X_b(s)^*, i.e.
    # conj F_ba) would change the density-velocity correlator by O(1): the statistical pin
    # above cannot pass with either mistake
    p = _params(lattice="D1Q3", nx=16, ny=1, tau=W.taus_d1q3(0.8), kT=1e-4, seed=1, init_mode=1, fields=[0, 9])
    ks = [(0, 1), (0, 2)]
    F = theory.time_correlators(p, p.fields, ks, 6, 1)
    assert np.abs(F[(0, 9)][1:] - np.conj(F[(0, 9)][1:])).max() > 0.5
    assert np.abs(F[(0, 9)][1:] - np.conj(F[(9, 0)][1:])).max() > 0.5
