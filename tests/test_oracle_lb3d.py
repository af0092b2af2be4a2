"""The three-dimensional lattices of the oracle (oracle.lb3d): D3Q15, which the paper
reports testing without printing its tables (Sec. 3), and D3Q19, both built from
Eqs. 2-5 and 8 and pinned against what the mathematics fixes (CPU only)."""
import numpy as np
import pytest

from oracle import lattice
from oracle import lb3d as D

LATS = ["D3Q15", "D3Q19"]


def _ng(name):
    return D.LATTICES[name].q - 10                 # ghost moments


@pytest.mark.parametrize("name", LATS)
def test_velocity_set_and_weights(name):
    L = D.LATTICES[name]
    v = L.v
    assert len({tuple(x) for x in v}) == L.q                     # distinct velocities
    for i in range(L.q):                                         # closed under v -> -v
        assert any(np.array_equal(-v[i], v[j]) for j in range(L.q))
    assert np.isclose(L.w.sum(), 1.0)
    assert np.abs((L.w[:, None] * v).sum(0)).max() < 1e-15
    assert np.abs((L.w[:, None, None] * v[:, :, None] * v[:, None, :]).sum(0) - np.eye(3) / 3).max() < 1e-15
    # the fourth moment is isotropic: sum w v_a v_b v_c v_d = (d_ab d_cd + d_ac d_bd + d_ad d_bc) / 9
    T = np.einsum("i,ia,ib,ic,id->abcd", L.w, v, v, v, v)
    I = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.abs(T - iso).max() < 1e-15


@pytest.mark.parametrize("name", LATS)
def test_orthonormal_complete_basis(name):
    L = D.LATTICES[name]
    G = (L.m * L.w[None, :]) @ L.m.T                           # Eq. 4
    assert np.abs(G - np.eye(L.q)).max() < 1e-14
    assert np.abs(L.m.T @ L.m * L.w[None, :] - np.eye(L.q)).max() < 1e-13     # completeness
    assert np.abs(L.n @ L.m - np.eye(L.q)).max() < 1e-13                        # n_i^a = w_i m_i^a inverts m


@pytest.mark.parametrize("name", LATS)
def test_moment_roles(name):
    L = D.LATTICES[name]
    v = L.v
    assert np.allclose(L.m[0], 1.0)
    assert np.allclose(L.m[1:4], np.sqrt(3.0) * v.T)           # momentum rows
    # every polynomial of degree <= 2 lies in the span of rows 0..9; the ghost rows are
    # orthogonal to all of them (hydrodynamic moments and ghosts decouple)
    polys = [np.ones(L.q)] + [v[:, a] for a in range(3)] + [v[:, a] * v[:, b] for a in range(3) for b in range(a, 3)]
    for P in polys:
        assert np.abs((L.m[10:] * L.w[None, :]) @ P).max() < 1e-14
        coef = (L.m[:10] * L.w[None, :]) @ P
        assert np.abs(L.m[:10].T @ coef - P).max() < 1e-13
    # the stress rows carry the second-order Hermite polynomials v_a v_b - delta_ab / 3
    H = [v[:, a] * v[:, b] - (a == b) / 3.0 for a in range(3) for b in range(a, 3)]
    S = np.array([(L.m[4:10] * L.w[None, :]) @ h for h in H])
    assert np.linalg.matrix_rank(S, tol=1e-10) == 6
    assert L.m.shape == (L.q, L.q) and len(L.nonconserved) == 6 + _ng(name)


@pytest.mark.parametrize("name", LATS)
def test_equilibrium_second_moments_exact(name):
    L = D.LATTICES[name]
    rho, u = 1.3, np.array([0.07, -0.05, 0.11])
    f0 = lattice.equilibrium(L, np.array(rho), u)
    assert np.isclose(f0.sum(), rho)
    assert np.allclose(L.v.T @ f0, rho * u)
    P = (f0[:, None, None] * L.v[:, :, None] * L.v[:, None, :]).sum(0)
    assert np.abs(P - rho * (np.eye(3) / 3 + np.outer(u, u))).max() < 1e-15
    # the ghost moments of f^0 vanish (f^0 / w is a polynomial of degree 2 in v)
    assert np.abs(L.m[10:] @ f0).max() < 1e-15


def _params(name, **kw):
    q = D.LATTICES[name].q
    d = dict(nx=8, ny=6, nz=4, tau=[1.0] * 4 + [0.8] * 6 + [1.1] * (q - 10), kT=1e-3, seed=3, lattice=name)
    d.update(kw)
    return D.Params3(**d)


@pytest.mark.parametrize("name", LATS)
def test_conservation_with_noise(name):
    r = D.Run3(_params(name, u0=(0.05, -0.02, 0.03), init_mode=1))
    c0 = r.conserved()
    r.run(12)
    assert np.abs(r.conserved() - c0).max() < 1e-12 * abs(c0[0])


@pytest.mark.parametrize("name", LATS)
def test_noise_statistics_of_one_step(name):
    # from the uniform equilibrium at tau = 1 the post-collision non-conserved moments are
    # exactly the noise: unit variance after dividing by sqrt(mu rho0), density and
    # momentum untouched
    q = D.LATTICES[name].q
    p = _params(name, nx=16, ny=16, nz=16, tau=[1.0] * q, kT=1e-2)
    L = D.LATTICES[name]
    f = D.collide(p, D.stream(D.uniform_state(p)), 5)
    dM = np.tensordot(L.m, f - D.uniform_state(p), axes=(1, 0)) / np.sqrt(p.mu * p.rho0)
    assert np.abs(dM[:4]).max() < 1e-12
    x = dM[4:].reshape(len(L.nonconserved), -1)
    assert np.abs(x.mean(1)).max() < 5 * 1 / np.sqrt(x.shape[1])
    assert np.abs(x.var(1) - 1).max() < 5 * np.sqrt(2 / x.shape[1])
    assert np.abs(np.corrcoef(x) - np.eye(len(x))).max() < 5 / np.sqrt(x.shape[1])


@pytest.mark.parametrize("name", LATS)
def test_shear_wave_decay(name):
    # u_x(y) = A sin(2 pi y / ny): decays per step by the factor of the linear operator,
    # close to exp(-nu k^2) with nu = (tau_s - 1/2) / 3
    q = D.LATTICES[name].q
    tau_s = 0.9
    p = _params(name, nx=4, ny=32, nz=4, tau=[1.0] * 4 + [tau_s] * 6 + [1.0] * (q - 10), kT=0.0)
    L = D.LATTICES[name]
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


@pytest.mark.parametrize("name", LATS)
def test_theory_flat_at_rest(name):
    p = _params(name, u0=(0.0, 0.0, 0.0), fields=[0, 1, 2, 3, 4, 10, D.LATTICES[name].q - 1])
    ks = [(0, 0, 1), (1, 2, 3), (3, 5, 7), (1, 0, 0)]
    assert np.all(np.isnan(D.point_theory(p, [0], [(2, 0, 0)])[(0, 0)]))      # k_z = pi: neutral
    C = D.point_theory(p, p.fields, ks)
    for (a, b), v in C.items():
        assert np.abs(v - (1.0 if a == b else 0.0)).max() < 1e-10, (a, b)
    # and not flat in a moving frame
    C = D.point_theory(_params(name, u0=(0.15, 0.0, 0.0), fields=[0, 1]), [0, 1], ks)
    assert np.abs(C[(0, 0)] - 1.0).max() > 1e-2


@pytest.mark.parametrize("name", LATS)
def test_simulated_spectra_match_theory(name):
    q = D.LATTICES[name].q
    p = _params(name, nx=6, ny=6, nz=4, tau=[1.0] * 4 + [0.8] * 6 + [1.0] * (q - 10), kT=1e-4,
                u0=(0.1, 0.0, 0.0), init_mode=1, fields=[0, 1, 4], seed=7)
    ks = [(0, 0, 1), (1, 2, 3), (1, 1, 2)]          # no component at pi (no neutral mode)
    C = D.point_theory(p, p.fields, ks)
    assert all(np.all(np.isfinite(v)) for v in C.values())
    r = D.Run3(p)
    r.run(200)
    batches = {pr: [] for pr in C}
    for _ in range(16):
        r.acc = D.PointAccumulator3(p, ks)
        r.run(200, 2)
        for pr in batches:
            batches[pr].append(r.acc.correlator(*pr))
    worst = 0.0
    for pr, v in batches.items():
        m, se = np.mean(v, 0), np.std(v, 0, ddof=1) / np.sqrt(len(v))
        for part in (np.real, np.imag):
            z = np.abs(part(m) - part(C[pr])) / np.maximum(se, 1e-3)
            assert np.all(np.isfinite(z))
            worst = max(worst, z.max())
    # 54 values of a t statistic with 15 degrees of freedom: P(max > 5) ~ 1e-2
    assert worst < 5.0, worst


def test_planted_ghost_amplitude_error_detected():
    # the batch-means statistic of test_simulated_spectra_match_theory rejects a run whose
    # noise on one ghost moment is 1.2 times the Eq. 8 amplitude (planted in the oracle)
    p = _params("D3Q19", nx=6, ny=6, nz=4, tau=[1.0] * 4 + [0.8] * 6 + [1.0] * 9, kT=1e-4, fields=[16], seed=2,
                init_mode=1)
    ks = [(0, 0, 1), (1, 2, 3), (1, 1, 2)]
    C = D.point_theory(p, p.fields, ks)[(16, 16)].real
    base = D.collide

    def planted(pp, f, t, return_parts=False):
        out, parts = base(pp, f, t, return_parts=True)
        L = pp.lat
        return out + 0.2 * np.tensordot(L.n[:, 16], parts["xi"][16], axes=0)

    D.collide = planted
    try:
        r = D.Run3(p)
        r.run(50)
        vals = []
        for _ in range(16):
            r.acc = D.PointAccumulator3(p, ks)
            r.run(200, 1)
            vals.append(r.acc.correlator(16, 16).real)
    finally:
        D.collide = base
    m, se = np.mean(vals, 0), np.std(vals, 0, ddof=1) / np.sqrt(len(vals))
    assert np.abs((m - C) / se).max() > 6.0, (m, C, se)
