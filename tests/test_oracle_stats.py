"""The oracle's simulated equal-time spectra against the exact linear theory (CPU only).

Batch means give a standard error per (k, pair); every included point must lie
within 5 standard errors of the theory.  The thermal start is the exact
stationary law at u0 = 0, so no warm-up is needed there.
"""
import numpy as np
import pytest

from oracle import lb, spectra, theory
from paper_1010_1233_gb300 import workloads as W

LADD = (1 << 3) | (1 << 4) | (1 << 5)


def _batch_spectra(p, n_batches, steps, warmup=0):
    r = lb.Run(p)
    r.run(warmup)
    out = {pr: [] for pr in spectra.pairs(p.fields)}
    for _ in range(n_batches):
        r.acc = spectra.Accumulator(p)
        r.run(steps, 1)
        for pr in out:
            out[pr].append(r.acc.correlator(*pr))
    return {pr: (np.mean(v, 0), np.std(v, 0, ddof=1) / np.sqrt(len(v))) for pr, v in out.items()}


def _check(p, meas, zmax=5.0, floor=1e-3):
    S, ex = theory.theory_spectra(p, p.fields)
    ok = ~ex
    worst = 0.0
    for pr, (m, se) in meas.items():
        for part in (np.real, np.imag):
            z = np.abs(part(m) - part(S[pr])) / np.maximum(se, floor)
            worst = max(worst, z[ok].max())
    assert worst < zmax, worst
    return S, ex


def _params(**kw):
    return lb.Params(**W.replica(**kw))


def test_d1q3_flat_spectra():
    p = _params(lattice="D1Q3", nx=16, ny=1, tau=W.taus_d1q3(0.8), kT=1e-4, seed=1,
                init_mode=1, fields=[0, 1])
    meas = _batch_spectra(p, 12, 1000)
    _check(p, meas)


def test_d2q9_ladd_spectra_match_theory():
    # ghost noise off at u0 = 0: strongly non-flat spectra, still predicted exactly
    p = _params(nx=8, ny=8, tau=W.taus_d2q9(1.0), kT=1e-4, seed=2, noise_mask=LADD,
                fields=[0, 9, 10])
    meas = _batch_spectra(p, 10, 600, warmup=200)
    S, ex = _check(p, meas)
    assert np.abs(S[(0, 0)] - 1)[~ex].max() > 0.3         # the comparison is non-trivial


def test_d2q9_moving_frame_matches_theory():
    # u0 = 0.15 with full ghost noise: Galilean-invariance violation of Sec. 3
    p = _params(nx=8, ny=8, tau=W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, seed=3, u0=(0.15, 0.0),
                init_mode=1, fields=[0, 9, 10])
    meas = _batch_spectra(p, 10, 600, warmup=300)
    _check(p, meas)


def test_planted_amplitude_mistake_is_detected(monkeypatch):
    # a 5 % error in the noise amplitude of the oracle must fail the spectral pin
    real = lb._rng.site_normals
    monkeypatch.setattr(lb._rng, "site_normals",
                        lambda n, *a, **k: real(n, *a, **k) * (1.05 if n < 9 else 1.0))
    p = _params(lattice="D1Q3", nx=16, ny=1, tau=W.taus_d1q3(0.8), kT=1e-4, seed=1,
                init_mode=1, fields=[0, 1])
    meas = _batch_spectra(p, 12, 1000)
    with pytest.raises(AssertionError):
        _check(p, meas)
