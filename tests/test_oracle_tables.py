"""Pins of the oracle's lattice tables against what Sec. 2-3 fix (CPU only)."""
import numpy as np
import pytest

from oracle import lattice as L


@pytest.mark.parametrize("lat", [L.D2Q9, L.D1Q3], ids=lambda l: l.name)
def test_hermite_orthonormality(lat):
    # Eq. 4: sum_i w_i m_i^a m_i^b = sum_i m_i^a n_i^b = delta^ab
    G = np.einsum("i,ai,bi->ab", lat.w, lat.m, lat.m)
    assert np.abs(G - np.eye(lat.q)).max() < 1e-15
    assert np.abs(lat.m @ lat.n - np.eye(lat.q)).max() < 1e-15
    # completeness: the back transform inverts the forward one
    assert np.abs(lat.n @ lat.m - np.eye(lat.q)).max() < 1e-15


@pytest.mark.parametrize("lat", [L.D2Q9, L.D1Q3], ids=lambda l: l.name)
def test_weights_and_velocity_moments(lat):
    # standard isothermal lattice: sum w = 1, sum w v = 0, sum w v v = 1/3 I
    assert abs(lat.w.sum() - 1) < 1e-15
    assert np.abs(lat.w @ lat.v).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", lat.w, lat.v, lat.v) - np.eye(lat.d) / 3).max() < 1e-15


def test_d2q9_velocities_as_printed():
    # Sec. 3 velocity list
    v = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    assert np.array_equal(L.D2Q9.v, np.array(v, dtype=float))


def test_d2q9_rows_are_hermite_polynomials():
    # Eq. 9 rows written as polynomials of v (shear, bulk and ghost identification of Sec. 3)
    v = L.D2Q9.v
    vx, vy = v[:, 0], v[:, 1]
    v2 = vx**2 + vy**2
    m = L.D2Q9.m
    assert np.allclose(m[1], np.sqrt(3) * vx) and np.allclose(m[2], np.sqrt(3) * vy)
    assert np.allclose(m[3], 1.5 * (vx**2 - vy**2)) and np.allclose(m[4], 3 * vx * vy)
    assert np.allclose(m[5], 1.5 * v2 - 1)
    assert np.allclose(m[6], np.sqrt(1.5) * vx * (3 * v2 - 4))
    assert np.allclose(m[7], np.sqrt(1.5) * vy * (3 * v2 - 4))


def test_equilibrium_moments_closed_forms():
    # Eq. 10 from the dense sum of Eq. 2
    rng = np.random.default_rng(0)
    rho = 1 + 0.1 * rng.standard_normal(50)
    u = 0.2 * rng.standard_normal((2, 50))
    M = L.D2Q9.m @ L.equilibrium(L.D2Q9, rho, u)
    ux, uy = u
    cf = np.array([rho, np.sqrt(3) * rho * ux, np.sqrt(3) * rho * uy,
                   1.5 * rho * (ux**2 - uy**2), 3 * rho * ux * uy, 1.5 * rho * (ux**2 + uy**2),
                   0 * rho, 0 * rho, 0 * rho])
    assert np.abs(M - cf).max() < 1e-15


def test_equilibrium_pressure_tensor():
    # Eq. 2 reproduces mass, momentum and the ideal-gas momentum flux rho (I/3 + u u)
    rng = np.random.default_rng(1)
    for lat in (L.D2Q9, L.D1Q3):
        rho = 1 + 0.1 * rng.standard_normal(20)
        u = 0.2 * rng.standard_normal((lat.d, 20))
        f = L.equilibrium(lat, rho, u)
        assert np.abs(f.sum(0) - rho).max() < 1e-14
        assert np.abs(lat.v.T @ f - rho * u).max() < 1e-14
        Pi = np.einsum("ia,ib,is->abs", lat.v, lat.v, f)
        want = rho * (np.eye(lat.d)[:, :, None] / 3 + u[:, None, :] * u[None, :, :])
        assert np.abs(Pi - want).max() < 1e-14


def test_d1q3_is_projection_of_d2q9():
    # Sec. 3: projecting D2Q9 onto one axis gives D1Q3
    w = {}
    for vi, wi in zip(L.D2Q9.v[:, 0], L.D2Q9.w):
        w[vi] = w.get(vi, 0) + wi
    for vi, wi in zip(L.D1Q3.v[:, 0], L.D1Q3.w):
        assert abs(w[vi] - wi) < 1e-15
    # the projected equilibrium of D2Q9 (u_y = 0) equals the D1Q3 equilibrium
    rho, ux = np.array([1.03]), np.array([[0.07], [0.0]])
    f2 = L.equilibrium(L.D2Q9, rho, ux)
    f1 = L.equilibrium(L.D1Q3, rho, ux[:1])
    for vi, fi in zip(L.D1Q3.v[:, 0], f1):
        assert abs(f2[L.D2Q9.v[:, 0] == vi].sum() - fi[0]) < 1e-15
    # D1Q3 stress moment of the equilibrium: 3 rho u^2 / sqrt 2
    M = L.D1Q3.m @ f1
    assert abs(M[2, 0] - 3 * 1.03 * 0.07**2 / np.sqrt(2)) < 1e-15
