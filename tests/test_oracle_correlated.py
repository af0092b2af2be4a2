"""Correlated noise for a moving fluid (oracle.correlated): pins (CPU only).

The extension follows the paper's remark after Eq. 7: with the global
equilibrium f^0(rho0, u0) in place of rho0 w the moment covariance is not
diagonal, and Eq. 6 asks for correlated noise on the non-conserved moments.
"""
import numpy as np
import pytest

from oracle import correlated, lattice, lb, spectra, theory
from paper_1010_1233_gb300 import workloads as W

D2Q9 = lattice.LATTICES["D2Q9"]
D1Q3 = lattice.LATTICES["D1Q3"]
LADD = (1 << 3) | (1 << 4) | (1 << 5)


def _all(lat):
    return sum(1 << a for a in lat.nonconserved)


@pytest.mark.parametrize("lat,tau,mask", [
    (D2Q9, W.taus_d2q9(0.8, 0.7, 1.3), None), (D2Q9, W.taus_d2q9(0.6, 0.6, 1.0), LADD),
    (D1Q3, W.taus_d1q3(0.55), None)])
def test_rest_frame_reduces_to_eq8(lat, tau, mask):
    mask = _all(lat) if mask is None else mask
    kT, rho0 = 1e-4, 1.3
    R, X, Xp = correlated.noise_root(lat, tau, rho0, kT, (0.0, 0.0), mask)
    mu = 3 * kT
    want = np.zeros(len(lat.nonconserved))
    for c, a in enumerate(lat.nonconserved):
        if (mask >> a) & 1:
            want[c] = np.sqrt(mu * rho0 * (2 * tau[a] - 1)) / tau[a]          # Eq. 8
    # (rounding of the dense moment sums and of the eigen-decomposition only)
    assert np.abs(R - np.diag(want)).max() < 1e-13 * want.max()
    assert np.abs(X - Xp).max() < 1e-13 * np.abs(X).max()


def test_moment_covariance_low_moments_closed_form():
    # mass, momentum and momentum flux of the discrete Maxwellian (Eq. 2) and the
    # equilibrium moments of Eq. 10 fix the first rows of C = mu sum m^a m^b f^0
    kT, rho0, (ux, uy) = 2e-4, 0.9, (0.23, -0.11)
    C = correlated.moment_covariance(D2Q9, rho0, kT, (ux, uy))
    mu, s3 = 3 * kT, np.sqrt(3.0)
    assert np.allclose(C[0, 0], mu * rho0, rtol=1e-14)
    assert np.allclose(C[0, 1:3], mu * rho0 * s3 * np.array([ux, uy]), rtol=1e-14)
    assert np.allclose(C[1, 1], mu * rho0 * (1 + 3 * ux * ux), rtol=1e-14)
    assert np.allclose(C[2, 2], mu * rho0 * (1 + 3 * uy * uy), rtol=1e-14)
    assert np.allclose(C[1, 2], mu * rho0 * 3 * ux * uy, rtol=1e-14)
    assert np.allclose(C[0, 3:6], mu * rho0 * np.array([1.5 * (ux * ux - uy * uy), 3 * ux * uy,
                                                         1.5 * (ux * ux + uy * uy)]), rtol=1e-13)
    assert np.abs(C - C.T).max() < 1e-15 * np.abs(C).max()
    assert np.linalg.eigvalsh(C).min() > 0


def test_root_and_positive_part():
    lat, kT = D2Q9, 1e-4
    # positive definite: X+ = X and R R = X on the non-conserved block
    tau = W.taus_d2q9(0.8, 0.8, 1.0)
    R, X, Xp = correlated.noise_root(lat, tau, 1.0, kT, (0.2, 0.05), _all(lat))
    nc = list(lat.nonconserved)
    assert np.abs(R - R.T).max() < 1e-14 * np.abs(R).max()
    assert np.abs(R @ R - X[np.ix_(nc, nc)]).max() < 1e-14 * np.abs(X).max()
    assert np.abs(Xp - X).max() < 1e-14 * np.abs(X).max()
    assert np.abs(X - np.diag(np.diag(X))).max() > 0.2 * np.abs(X).max()     # really correlated
    # indefinite (tau far apart, large u0): X+ drops exactly the negative eigenvalues
    tau = W.taus_d2q9(0.55, 0.55, 1.5)
    R, X, Xp = correlated.noise_root(lat, tau, 1.0, kT, (0.3, 0.1), _all(lat))
    w = np.linalg.eigvalsh(X[np.ix_(nc, nc)])
    assert w.min() < 0
    assert np.linalg.eigvalsh(Xp[np.ix_(nc, nc)]).min() > -1e-18
    assert np.isclose(np.linalg.norm(Xp - X), np.sqrt(np.sum(w[w < 0] ** 2)), rtol=1e-10)
    assert np.abs(R @ R - Xp[np.ix_(nc, nc)]).max() < 1e-14 * np.abs(X).max()


def test_step_samples_the_covariance_and_conserves():
    p = lb.Params(**W.replica("D2Q9", 64, 64, W.taus_d2q9(0.8, 0.7, 1.0), kT=1e-4, u0=(0.2, 0.05),
                              seed=5, noise_mode=1))
    f0 = lb.uniform_state(p)
    xs = []
    for t in range(8):
        _, parts = lb.collide(p, f0, t, return_parts=True)
        xs.append(parts["xi"][list(D2Q9.nonconserved)].reshape(6, -1))
    x = np.concatenate(xs, axis=1)
    n = x.shape[1]
    cov = x @ x.T / n
    _, _, Xp = correlated.noise_root(D2Q9, p.tau, p.rho0, p.kT, p.u0_vec(), p.mask())
    B = Xp[np.ix_(list(D2Q9.nonconserved), list(D2Q9.nonconserved))]
    se = np.sqrt((np.outer(np.diag(B), np.diag(B)) + B * B) / n)
    assert np.abs(cov - B).max() / se.max() < 5.0
    # density and momentum untouched by the noise
    r = lb.Run(p)
    m0 = r.conserved()
    r.run(5)
    # (up to the rounding of sums over 64^2 sites of size ~1: V eps per step)
    assert np.abs(np.asarray(r.conserved()) - np.asarray(m0)).max() < 5 * 64 * 64 * 2.2e-16


def test_theory_rest_frame_flat_and_moving_frame_improved():
    kw = dict(nx=12, ny=12, tau=W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, fields=[0, 9, 10])
    p0 = lb.Params(**W.replica(u0=(0.0, 0.0), noise_mode=1, **kw))
    S, ex = theory.theory_spectra(p0, p0.fields)
    for (a, b), v in S.items():
        want = 1.0 if a == b else 0.0
        assert np.abs(v[~ex] - want).max() < 1e-9
    # at u0 = 0.1 the correlated noise removes most of the violation of the flat spectra
    errs = {}
    for mode in (0, 1):
        p = lb.Params(**W.replica(u0=(0.1, 0.0), noise_mode=mode, **kw))
        S, ex = theory.theory_spectra(p, p.fields)
        errs[mode] = np.mean([np.abs(v[~ex] - (1.0 if a == b else 0.0)).mean() for (a, b), v in S.items()])
    assert errs[1] < 0.5 * errs[0], errs


def test_oracle_simulation_matches_correlated_theory():
    # simulated spectra with the correlated noise against the linear theory
    from test_oracle_stats import _batch_spectra, _check
    p = lb.Params(**W.replica(nx=8, ny=8, tau=W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, seed=13, u0=(0.15, 0.0),
                              init_mode=1, fields=[0, 9, 10], noise_mode=1))
    meas = _batch_spectra(p, 10, 600, warmup=300)
    _check(p, meas)


def test_independent_noise_fails_the_correlated_pin():
    # planted mistake: the diagonal scheme measured against the correlated theory
    import dataclasses
    from test_oracle_stats import _batch_spectra, _check
    p = lb.Params(**W.replica(nx=8, ny=8, tau=W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, seed=13, u0=(0.15, 0.0),
                              init_mode=1, fields=[0, 9, 10], noise_mode=0))
    meas = _batch_spectra(p, 10, 600, warmup=300)
    with pytest.raises(AssertionError):
        _check(dataclasses.replace(p, noise_mode=1), meas)
