"""Correlated noise for a moving fluid, FP64 (test infrastructure only).

An extension the paper points to but does not build (Sec. 2, after Eq. 7): the
decoupling of the moment fluctuations, <dM^a dM^b> = rho-bar delta^ab, uses
f-bar_i = rho-bar w_i, i.e. u << 1.  For a fluid at rest in a frame moving with
the mean velocity u0 the global equilibrium is f-bar = f^0(rho0, u0) of Eq. 2,
and the same sum gives a non-diagonal covariance

    C_ab = mu sum_i m_i^a m_i^b f^0_i(rho0, u0)                    (Eq. 7, first lines)

(mu = 3 k_B T as in the diagonal scheme).  The fluctuation-dissipation relation of
Eq. 6 then asks for correlated noise on the non-conserved moments,

    <xi^a xi^c> = (tau^a + tau^c - 1) / (tau^a tau^c) C_ac,   a, c non-conserved and in the mask,

and zero noise on density and momentum.  This matrix need not be positive
semi-definite (for tau^a far apart at large u0); the noise uses its positive part
(eigenvalues below zero set to zero), and xi = R N with R the principal (symmetric)
square root of that part and N the site's unit normals in the order of the
non-conserved moments.  At u0 = 0, C = mu rho0 I and R is the diagonal of Eq. 8.

Parity: pinned by the u0 = 0 reduction to Eq. 8, by the closed-form low moments of
the discrete Maxwellian (mass, momentum and the momentum-flux tensor of Eq. 2), by
R R = positive part, and by the sampled covariance of xi in the oracle's step.
"""
import numpy as np

from . import lattice as _lat


def moment_covariance(lat, rho0, kT, u0):
    """C_ab = mu sum_i m_i^a m_i^b f^0_i(rho0, u0), shape (q, q)."""
    u = np.asarray(u0, dtype=np.float64)[: lat.d]
    fbar = _lat.equilibrium(lat, np.array(float(rho0)), u)
    return 3.0 * kT * (lat.m * fbar[None, :]) @ lat.m.T


def noise_covariance(lat, tau, rho0, kT, u0, mask):
    """<xi^a xi^c> of Eq. 6 with the covariance above on the masked non-conserved moments."""
    C = moment_covariance(lat, rho0, kT, u0)
    tau = np.asarray(tau, dtype=np.float64)
    act = [a for a in lat.nonconserved if (mask >> a) & 1]
    X = np.zeros((lat.q, lat.q))
    for a in act:
        for c in act:
            X[a, c] = (tau[a] + tau[c] - 1.0) / (tau[a] * tau[c]) * C[a, c]
    return X


def noise_root(lat, tau, rho0, kT, u0, mask):
    """(R, X, X+): R the principal square root of X+ on the non-conserved block,
    shape (n_nc, n_nc) in the order of lat.nonconserved; X the matrix of Eq. 6
    (q x q); X+ its positive part (q x q)."""
    X = noise_covariance(lat, tau, rho0, kT, u0, mask)
    nc = list(lat.nonconserved)
    B = X[np.ix_(nc, nc)]
    w, V = np.linalg.eigh(B)
    wp = np.clip(w, 0.0, None)
    R = (V * np.sqrt(wp)[None, :]) @ V.T
    Xp = np.zeros_like(X)
    Xp[np.ix_(nc, nc)] = (V * wp[None, :]) @ V.T
    return R, X, Xp
