"""D3Q15 (oracle.d3q15): the lattice the paper reports testing without printing its
tables (Sec. 3), built from Eqs. 2-5 and 8 and pinned (CPU only)."""
import numpy as np
import pytest

from oracle import d3q15 as D
from oracle import lattice

L = D.LATTICE


def test_orthonormal_complete_basis():
    G = (L.m * L.w[None, :]) @ L.m.T                           # Eq. 4
    assert np.abs(G - np.eye(15)).max() < 1e-14
    assert np.abs(L.m.T @ L.m * L.w[None, :] - np.eye(15)).max() < 1e-13     # completeness
    assert np.allclose(L.w.sum(), 1.0) and np.allclose((L.w[:, None, None] * L.v[:, :, None] * L.v[:, None, :]).sum(0),
                                                       np.eye(3) / 3)


def test_moment_roles():
    v = L.v
    assert np.allclose(L.m[0], 1.0)
    assert np.allclose(L.m[1:4], np.sqrt(3.0) * v.T)           # momentum rows
    # every polynomial of degree <= 2 lies in the span of rows 0..9; the ghost rows are
    # orthogonal to all of them (hydrodynamic moments and ghosts decouple)
    polys = [np.ones(15)] + [v[:, a] for a in range(3)] + [v[:, a] * v[:, b] for a in range(3) for b in range(a, 3)]
    for P in polys:
        assert np.abs((L.m[10:] * L.w[None, :]) @ P).max() < 1e-14
        coef = (L.m[:10] * L.w[None, :]) @ P
        assert np.abs(L.m[:10].T @ coef - P).max() < 1e-13
    # the stress rows carry the second-order Hermite polynomials v_a v_b - delta_ab / 3
    H = [v[:, a] * v[:, b] - (a == b) / 3.0 for a in range(3) for b in range(a, 3)]
    S = np.array([(L.m[4:10] * L.w[None, :]) @ h for h in H])
    assert np.linalg.matrix_rank(S, tol=1e-10) == 6


def test_equilibrium_second_moments_exact():
    rho, u = 1.3, np.array([0.07, -0.05, 0.11])
    f0 = lattice.equilibrium(L, np.array(rho), u)
    assert np.isclose(f0.sum(), rho)
    assert np.allclose(L.v.T @ f0, rho * u)
    P = (f0[:, None, None] * L.v[:, :, None] * L.v[:, None, :]).sum(0)
    assert np.abs(P - rho * (np.eye(3) / 3 + np.outer(u, u))).max() < 1e-15


def _params(**kw):
    d = dict(nx=8, ny=6, nz=4, tau=[1.0] * 4 + [0.8] * 6 + [1.1] * 5, kT=1e-3, seed=3)
    d.update(kw)
    return D.Params3(**d)


def test_conservation_with_noise():
    r = D.Run3(_params(u0=(0.05, -0.02, 0.03), init_mode=1))
    c0 = r.conserved()
    r.run(12)
    assert np.abs(r.conserved() - c0).max() < 1e-12 * abs(c0[0])


def test_shear_wave_decay():
    # u_x(y) = A sin(2 pi y / ny): decays per step by the factor of the linear operator,
    # close to exp(-nu k^2) with nu = (tau_s - 1/2) / 3
    tau_s = 0.9
    p = _params(nx=4, ny=32, nz=4, tau=[1.0] * 4 + [tau_s] * 6 + [1.0] * 5, kT=0.0)
    y = np.arange(p.ny)
    A = 1e-6
    ux = np.broadcast_to((A * np.sin(2 * np.pi * y / p.ny))[None, :, None], (p.nz, p.ny, p.nx))
    u = np.stack([ux, np.zeros_like(ux), np.zeros_like(ux)])
    f = lattice.equilibrium(L, np.ones((p.nz, p.ny, p.nx)), u)
    amps = []
    for _ in range(40):
        f = D.collide(p, D.stream(f), 0)
        _, _, uu = D.macroscopic(f)
        amps.append(np.abs(np.fft.fft(uu[0, 0, :, 0]))[1])
    rate = -np.log(amps[-1] / amps[-21]) / 20
    k = 2 * np.pi / p.ny
    nu = (tau_s - 0.5) / 3
    assert abs(rate - nu * k * k) < 2e-3 * nu * k * k + 1e-6


def test_theory_flat_at_rest():
    p = _params(u0=(0.0, 0.0, 0.0), fields=[0, 1, 2, 3, 4, 10])
    ks = [(0, 0, 1), (1, 2, 3), (3, 5, 7), (1, 0, 0)]
    assert np.all(np.isnan(D.point_theory(p, [0], [(2, 0, 0)])[(0, 0)]))      # k_z = pi: neutral
    C = D.point_theory(p, p.fields, ks)
    for (a, b), v in C.items():
        assert np.abs(v - (1.0 if a == b else 0.0)).max() < 1e-10, (a, b)
    # and not flat in a moving frame
    C = D.point_theory(_params(u0=(0.15, 0.0, 0.0), fields=[0, 1]), [0, 1], ks)
    assert np.abs(C[(0, 0)] - 1.0).max() > 1e-2


def test_simulated_spectra_match_theory():
    p = _params(nx=6, ny=6, nz=4, tau=[1.0] * 4 + [0.8] * 6 + [1.0] * 5, kT=1e-4, u0=(0.1, 0.0, 0.0),
                init_mode=1, fields=[0, 1, 4], seed=7)
    ks = [(0, 0, 1), (1, 2, 3), (2, 3, 0)]
    C = D.point_theory(p, p.fields, ks)
    r = D.Run3(p)
    r.run(200)
    batches = {pr: [] for pr in C}
    for _ in range(8):
        r.acc = D.PointAccumulator3(p, ks)
        r.run(400, 2)
        for pr in batches:
            batches[pr].append(r.acc.correlator(*pr))
    worst = 0.0
    for pr, v in batches.items():
        m, se = np.mean(v, 0), np.std(v, 0, ddof=1) / np.sqrt(len(v))
        for part in (np.real, np.imag):
            worst = max(worst, (np.abs(part(m) - part(C[pr])) / np.maximum(se, 1e-3)).max())
    assert worst < 5.0, worst
