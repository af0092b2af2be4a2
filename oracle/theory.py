"""Linear theory of the fluctuating step (test infrastructure only).

For small fluctuations around the uniform state f-bar = f^0(rho0, u0) the step
of ``oracle.lb`` is linear in Fourier space:

    df(k, t+1) = A_k df(k, t) + P_k N xi(k, t),    A_k = P_k J,

where P_k = diag(exp(-i k.v_i)) is the pull streaming (Eq. 1), J is the
derivative of the collision (Eq. 5) with respect to the pre-collision f,

    J = N [ (I - T) M + T M F ],   T = diag(1/tau^a on non-conserved a, 0 on conserved a),
    F_ij = d f_i^0 / d f_j of Eq. 2 at (rho0, u0),

(M = m_i^a of Eq. 9, N = n_i^a = w_i m_i^a), and xi is white noise with per-site
variances sigma_a^2 = s_a^2 mu rho0 (2 tau^a - 1) / tau_a^2 (Eq. 8), or with the
covariance of the correlated scheme (``noise_matrix``).  The
stationary equal-time covariance per unit volume C_k = <df(k) df(k)^H> / V then
solves the discrete Lyapunov equation

    C_k = A_k C_k A_k^H + P_k N diag(sigma^2) N^T P_k^H,

and a linear field X = L df has <X_a(k) X_b(k)^*> / V = (L C_k L^H)_ab.  At
u0 = 0 with noise on every non-conserved moment its solution is C_k = mu rho0
diag(w) for every k, i.e. Eq. 7: <dM^a dM^b> = mu rho0 delta^ab.  With the ghost
noise off, or at u0 != 0, it gives the non-trivial spectra of Figs. 1-4.

Wave vectors where A_k has an eigenvalue of unit modulus (k = 0, where density
and momentum are conserved, and lattice-specific neutral modes such as
k = (pi, 0) for D2Q9 or k = pi for D1Q3, where a momentum component only flips
sign every step and receives no noise) have no unique stationary state; they
are flagged and excluded.

Parity: pinned by Eq. 7 (u0 = 0, full noise: S = delta_ab to rounding), by the
paper's statement that the Ladd scheme has no deficiency on the k_x = 0 and
k_y = 0 axes (Sec. 3), by its printed maximal Ladd cross correlation (~0.25,
Sec. 3), and by the oracle simulation (tiny-amplitude waves follow A_k exactly;
measured spectra agree within statistical error).
"""
import numpy as np
import scipy.linalg as sla

from . import correlated as _corr
from . import lattice as _lat


def equilibrium_jacobian(lat, rho0, u0):
    """F_ij = d f_i^0 / d f_j at (rho0, u0), from Eq. 2 written in (rho, j = rho u)."""
    u0 = np.asarray(u0, dtype=np.float64)[: lat.d]
    uv = lat.v @ u0                                     # (q,)
    uu = float(u0 @ u0)
    d_rho = lat.w * (1.0 - 4.5 * uv**2 + 1.5 * uu)      # d f_i^0 / d rho
    d_j = lat.w[:, None] * (3.0 * lat.v + 9.0 * uv[:, None] * lat.v - 3.0 * u0[None, :])  # (q, d)
    # d rho / d f_j = 1 ; d j_alpha / d f_j = v_j,alpha
    return d_rho[:, None] * np.ones((1, lat.q)) + d_j @ lat.v.T


def collision_jacobian(lat, tau, rho0, u0):
    T = np.zeros(lat.q)
    for a in lat.nonconserved:
        T[a] = 1.0 / tau[a]
    F = equilibrium_jacobian(lat, rho0, u0)
    return lat.n @ ((np.eye(lat.q) - np.diag(T)) @ lat.m + np.diag(T) @ lat.m @ F)


def noise_variances(lat, tau, rho0, kT, mask, scale=None):
    """sigma_a^2 of Eq. 8 (times s_a^2), zero on conserved and masked moments."""
    mu = 3.0 * kT
    s2 = np.zeros(lat.q)
    for c, a in enumerate(lat.nonconserved):
        if (mask >> a) & 1:
            s = 1.0 if scale is None else float(scale[c])
            s2[a] = s * s * mu * rho0 * (2.0 * tau[a] - 1.0) / tau[a] ** 2
    return s2


def noise_matrix(p, scale=None):
    """Covariance of the moment noise xi (q x q): diag(sigma^2) of Eq. 8, or for
    p.noise_mode == 1 the positive part of Eq. 6 at u0 (oracle.correlated); the
    per-moment scales s multiply rows and columns."""
    lat = p.lat
    tau = np.asarray(p.tau, dtype=np.float64)
    if getattr(p, "noise_mode", 0) != 1:
        return np.diag(noise_variances(lat, tau, p.rho0, p.kT, p.mask(), scale))
    _, _, Xp = _corr.noise_root(lat, tau, p.rho0, p.kT, p.u0_vec(), p.mask())
    s = np.ones(lat.q)
    if scale is not None:
        for c, a in enumerate(lat.nonconserved):
            s[a] = float(scale[c])
    return s[:, None] * Xp * s[None, :]


def wavevectors(nx, ny):
    kx = 2.0 * np.pi * np.arange(nx) / nx
    ky = 2.0 * np.pi * np.arange(ny) / ny
    return kx, ky


def streaming_phase(lat, kvec):
    return np.exp(-1j * (lat.v @ np.asarray(kvec[: lat.d])))


def one_step_operator(lat, tau, rho0, u0, kvec):
    return streaming_phase(lat, kvec)[:, None] * collision_jacobian(lat, tau, rho0, u0)


def field_rows(p, fields):
    """Rows L_a of the linearised maps df -> dX_a (moment fields and velocity components)."""
    lat = p.lat
    u0 = p.u0_vec()
    rows = []
    for fid in fields:
        if fid < lat.q:
            rows.append(lat.m[fid])
        elif fid in (9, 10):
            al = fid - 9
            rows.append((lat.v[:, al] - u0[al]) / p.rho0)     # du = (dj - u0 drho) / rho0
        else:
            raise ValueError(fid)
    return np.array(rows)


def theory_spectra(p, fields, scale=None, tol=1e-9):
    """Predicted normalised C_ab(k) for every field pair and k on the (ny, nx) grid.

    Returns (S, excluded): S[(a, b)] complex (ny, nx); excluded boolean (ny, nx)
    marks k with an eigenvalue of A_k within tol of the unit circle.
    """
    from .spectra import field_variance, pairs
    lat = p.lat
    ny = p.ny if lat.d == 2 else 1
    nx = p.nx
    tau = np.asarray(p.tau, dtype=np.float64)
    J = collision_jacobian(lat, tau, p.rho0, p.u0_vec())
    Qf = lat.n @ noise_matrix(p, scale) @ lat.n.T
    L = field_rows(p, fields)
    var = np.array([field_variance(p, f) for f in fields])
    kx, ky = wavevectors(nx, ny)
    S = {pr: np.zeros((ny, nx), dtype=np.complex128) for pr in pairs(fields)}
    excluded = np.zeros((ny, nx), dtype=bool)
    idx = {f: i for i, f in enumerate(fields)}
    for iy in range(ny):
        for ix in range(nx):
            kvec = np.array([kx[ix], ky[iy]])
            P = streaming_phase(lat, kvec)
            A = P[:, None] * J
            lam = np.abs(np.linalg.eigvals(A))
            if lam.max() > 1.0 - tol:
                excluded[iy, ix] = True
                continue
            Q = (P[:, None] * Qf) * np.conj(P)[None, :]
            C = sla.solve_discrete_lyapunov(A, Q)
            G = L @ C @ L.conj().T
            for (a, b) in S:
                ia, ib = idx[a], idx[b]
                S[(a, b)][iy, ix] = G[ia, ib] / np.sqrt(var[ia] * var[ib])
    return S, excluded


def spectral_radius(p):
    """max over k of |eig(A_k)| (> 1 means linearly unstable)."""
    lat = p.lat
    ny = p.ny if lat.d == 2 else 1
    J = collision_jacobian(lat, np.asarray(p.tau, dtype=np.float64), p.rho0, p.u0_vec())
    kx, ky = wavevectors(p.nx, ny)
    r = 0.0
    for iy in range(ny):
        for ix in range(p.nx):
            P = streaming_phase(lat, np.array([kx[ix], ky[iy]]))
            r = max(r, np.abs(np.linalg.eigvals(P[:, None] * J)).max())
    return r


def time_correlators(p, fields, kpoints, n_lags, every, scale=None):
    """Predicted normalised F_ab(k, tau) = <X_a(k, s) X_b(k, s - tau)^*> (time
    correlators of spectra.TimeAccumulator) for lags of tau * every steps:
    the stationary covariance C_k propagated by the one-step operator,
    <df(k, t + m) df(k, t)^H> / V = A_k^m C_k.  Returns {(a, b): (n_lags, n_k)}."""
    from .spectra import field_variance
    lat = p.lat
    tau_m = np.asarray(p.tau, dtype=np.float64)
    J = collision_jacobian(lat, tau_m, p.rho0, p.u0_vec())
    Qf = lat.n @ noise_matrix(p, scale) @ lat.n.T
    L = field_rows(p, fields)
    var = np.array([field_variance(p, f) for f in fields])
    ny = p.ny if lat.d == 2 else 1
    out = {(a, b): np.zeros((n_lags, len(kpoints)), complex) for a in fields for b in fields}
    for j, (ky, kx) in enumerate(kpoints):
        kvec = np.array([2 * np.pi * kx / p.nx, 2 * np.pi * ky / ny])
        P = streaming_phase(lat, kvec)
        A = P[:, None] * J
        Q = (P[:, None] * Qf) * np.conj(P)[None, :]
        C = sla.solve_discrete_lyapunov(A, Q)
        Ae = np.linalg.matrix_power(A, int(every))
        G = C
        for t in range(n_lags):
            H = L @ G @ L.conj().T
            for ia, a in enumerate(fields):
                for ib, b in enumerate(fields):
                    out[(a, b)][t, j] = H[ia, ib] / np.sqrt(var[ia] * var[ib])
            G = Ae @ G
    return out

