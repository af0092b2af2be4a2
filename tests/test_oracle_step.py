"""Pins of the oracle's step (Eqs. 1-5, 8) against conservation laws and hydrodynamics (CPU only)."""
import numpy as np
import pytest

from oracle import lattice as L, lb, philox, theory
from paper_1010_1233_gb300 import workloads as W


def _params(**kw):
    d = W.replica(**kw)
    d.pop("fields")
    return lb.Params(**d)


def _perturbed(p, amp, seed):
    f = lb.uniform_state(p)
    return f * (1.0 + W.random_perturbation(f.shape, seed, amp))


@pytest.mark.parametrize("lattice,nx,ny", [("D2Q9", 12, 8), ("D1Q3", 16, 1)])
def test_mass_and_momentum_conserved_with_noise(lattice, nx, ny):
    # Sec. 2: the noise has no density or momentum component, so both are exact invariants
    tau = W.taus_d2q9(0.7, 0.9, 1.3) if lattice == "D2Q9" else W.taus_d1q3(0.7)
    p = _params(lattice=lattice, nx=nx, ny=ny, tau=tau, kT=1e-2, u0=(0.05, -0.03), seed=3)
    r = lb.Run(p, _perturbed(p, 0.05, 1))
    c0 = r.conserved()
    r.run(60)
    assert np.abs(r.conserved() - c0).max() < 1e-13 * nx * ny


def test_streaming_moves_each_population_along_its_velocity():
    p = _params(nx=7, ny=5)
    f = np.zeros((9, 5, 7))
    f[:, 2, 3] = 1.0
    g = lb.stream(p.lat, f)
    for i, (vx, vy) in enumerate(p.lat.v.astype(int)):
        assert g[i, (2 + vy) % 5, (3 + vx) % 7] == 1.0 and g[i].sum() == 1.0


def test_uniform_equilibrium_is_fixed_point():
    p = _params(tau=W.taus_d2q9(0.6, 0.8, 1.2), u0=(0.2, -0.1), noise_mask=0, nx=6, ny=4)
    r = lb.Run(p)
    f0 = r.f.copy()
    r.run(5)
    assert np.abs(r.f - f0).max() < 1e-15


def test_unit_tau_without_noise_returns_equilibrium():
    # tau^a = 1: every non-conserved moment is replaced by its equilibrium value,
    # and by completeness of the moment basis f* = f^0(rho, u) of Eq. 2
    p = _params(noise_mask=0, nx=6, ny=5)
    f = _perturbed(p, 0.1, 2)
    fstar = lb.collide(p, f, 0)
    rho, j, u = lb.macroscopic(p.lat, f)
    assert np.abs(fstar - L.equilibrium(p.lat, rho, u)).max() < 1e-15


def test_ladd_mask_leaves_ghost_moments_noise_free():
    # Sec. 3: the Ladd scheme = no noise on M^6..M^8; they relax deterministically
    tau = W.taus_d2q9(0.8, 0.8, 1.4)
    p = _params(tau=tau, noise_mask=(1 << 3) | (1 << 4) | (1 << 5), kT=0.1, nx=5, ny=4)
    f = _perturbed(p, 0.1, 4)
    fstar, parts = lb.collide(p, f, 3, return_parts=True)
    M = p.lat.m @ fstar.reshape(9, -1)
    Mb = parts["M"].reshape(9, -1)
    Mq = parts["Meq"].reshape(9, -1)
    for a in (6, 7, 8):
        assert np.abs(M[a] - (Mb[a] - (Mb[a] - Mq[a]) / tau[a])).max() < 1e-14
    assert np.abs(parts["xi"][3:6]).min() > 0


def test_noise_uses_generator_normals_per_moment():
    # the D2Q9 noise of moment 3 + c is normal c of the site's Philox draw (step t, tag 0)
    p = _params(tau=W.taus_d2q9(1.0), kT=0.2, nx=4, ny=3, seed=9, stream=2)
    f = lb.uniform_state(p)
    _, parts = lb.collide(p, f, 5, return_parts=True)
    N = philox.pair_normals(lb.site_index(p), 5, 0, 2, 9)
    assert np.abs(parts["xi"][3:] - np.sqrt(3 * 0.2) * N).max() < 1e-14


def _shear_run(L_, tau_s, steps, amp=1e-6):
    p = _params(nx=L_, ny=2, tau=W.taus_d2q9(tau_s, tau_s, 1.0), noise_mask=0)
    x = np.arange(L_)
    uy = amp * np.sin(2 * np.pi * x / L_)[None, :] * np.ones((2, 1))
    u = np.stack([np.zeros_like(uy), uy])
    f = L.equilibrium(p.lat, np.ones((2, L_)), u)
    r = lb.Run(p, f)
    k = 2 * np.pi / L_
    amps = []
    for t in range(steps + 1):
        if t:
            r.run(1)
        _, j, _ = lb.macroscopic(p.lat, lb.stream(p.lat, r.f))
        amps.append(np.sum(j[1, 0] * np.exp(-1j * k * x)))
    return p, f, np.array(amps)


def test_shear_wave_decays_at_continuum_viscosity():
    # nu = (tau_s - 1/2) / 3 in lattice units; amplitude ~ exp(-nu k^2 t)
    L_, tau_s = 64, 0.6
    _, _, a = _shear_run(L_, tau_s, 240)
    k = 2 * np.pi / L_
    rate = -np.log(abs(a[240]) / abs(a[40])) / 200
    nu = (tau_s - 0.5) / 3
    assert abs(rate / (nu * k * k) - 1) < 1e-3


def test_shear_wave_follows_exact_linear_operator():
    # tiny amplitude: the nonlinear oracle step equals A_k (analytic Jacobian) to O(amp)
    L_, tau_s = 16, 0.7
    p, f, a = _shear_run(L_, tau_s, 30)
    k = 2 * np.pi / L_
    A = theory.one_step_operator(p.lat, np.asarray(p.tau), 1.0, (0, 0), np.array([k, 0.0]))
    df0 = np.sum((lb.stream(p.lat, f) - lb.uniform_state(p))[:, 0, :]
                 * np.exp(-1j * k * np.arange(L_))[None, :], axis=1)
    vy = p.lat.v[:, 1]
    d = df0.copy()
    pred = []
    for t in range(31):
        pred.append(vy @ d)
        d = A @ d
    pred = np.array(pred)
    assert np.abs(a - pred).max() < 1e-5 * np.abs(pred).max()
