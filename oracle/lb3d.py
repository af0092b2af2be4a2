"""Three-dimensional fluctuating lattice Boltzmann steps of the oracle, FP64 (test infrastructure only).

The paper reports that it also tested D3Q15 (Sec. 3) without printing its tables, and
D3Q19 is the other standard three-dimensional lattice.  This module builds the scheme
of Sec. 2 on both from the same ingredients:

* velocities and weights (Sec. 3 style, sum_i w_i v_i v_i = delta / 3 as Eq. 2 needs):
  D3Q15: the rest vector (2/9), the six (+-1, 0, 0) and permutations (1/9), the eight
  (+-1, +-1, +-1) (1/72);
  D3Q19: the rest vector (1/3), the six axis vectors (1/18), the twelve (+-1, +-1, 0)
  and permutations (1/36);
* moments: an orthonormal basis in the weighted norm of Eq. 4, sum_i w_i m_i^a m_i^b
  = delta^ab, built by Gram-Schmidt from a list of polynomials in v taken in order:
      1, vx, vy, vz,                                                   (density, momentum)
      vx^2 - vy^2, vx^2 + vy^2 - 2 vz^2, vx vy, vy vz, vz vx, v^2,     (stress)
  then the ghosts,
      D3Q15: vx v^2, vy v^2, vz v^2, vx vy vz, v^4
      D3Q19: vx v^2, vy v^2, vz v^2, vx (vy^2 - vz^2), vy (vz^2 - vx^2), vz (vx^2 - vy^2),
             v^4, (vx^2 - vy^2) v^2, (vx^2 + vy^2 - 2 vz^2) v^2;
  a = 0 density, 1-3 momentum (times sqrt 3), 4-8 shear stress, 9 bulk stress, the rest
  ghost moments;
* equilibrium: f^0 of Eq. 2 with three velocity components;
* collision: Eq. 5 on the non-conserved moments, noise of Eq. 8 on each (unit normals
  from Philox4x32-10, calls 0, 1, ... of the counter (site, step, call, stream); normal
  c drives moment 4 + c), density and momentum untouched;
* pull streaming in x, y and z (periodic); the site index is (z ny + y) nx + x;
* the thermal start draws q moment normals per site with tag 1.

Sampled fields are moments (field id a < q) minus their reference value M^{a,0}(rho0,
u0); their transforms are direct sums at chosen wave vectors (Eq. 11), normalised by
1 / (V mu rho0) as in ``oracle.spectra``.

Parity: pinned per lattice by the orthonormality and completeness of the basis, the
moment roles (momentum rows, stress rows spanning the second-order Hermite polynomials,
ghosts orthogonal to every polynomial of degree <= 2), the exact second moments of f^0,
conservation with noise, shear-wave decay at nu = (tau - 1/2)/3, the flat equal-time
spectra of the linear theory at u0 = 0, and simulated spectra against that theory.
"""
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

from . import lattice as _lat
from . import philox as _rng

V15 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
       (1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1), (1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1)]
W15 = [2 / 9] + [1 / 9] * 6 + [1 / 72] * 8

# D3Q19: rest, +-x, +-y, +-z, then the xy, xz and yz edges, each as (+,+), (-,-), (+,-), (-,+)
V19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
       (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
       (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
       (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
W19 = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12


def _hydro(v):
    vx, vy, vz = v[:, 0], v[:, 1], v[:, 2]
    v2 = vx * vx + vy * vy + vz * vz
    return [np.ones_like(vx), vx, vy, vz,
            vx * vx - vy * vy, vx * vx + vy * vy - 2 * vz * vz, vx * vy, vy * vz, vz * vx, v2]


def _ghosts15(v):
    vx, vy, vz = v[:, 0], v[:, 1], v[:, 2]
    v2 = vx * vx + vy * vy + vz * vz
    return [vx * v2, vy * v2, vz * v2, vx * vy * vz, v2 * v2]


def _ghosts19(v):
    vx, vy, vz = v[:, 0], v[:, 1], v[:, 2]
    v2 = vx * vx + vy * vy + vz * vz
    return [vx * v2, vy * v2, vz * v2, vx * (vy * vy - vz * vz), vy * (vz * vz - vx * vx), vz * (vx * vx - vy * vy),
            v2 * v2, (vx * vx - vy * vy) * v2, (vx * vx + vy * vy - 2 * vz * vz) * v2]


def basis(v, w, polys):
    """Gram-Schmidt of the polynomial list in the weighted inner product of Eq. 4."""
    rows = []
    for p in polys:
        r = np.asarray(p, dtype=np.float64).copy()
        for q in rows:
            r -= np.sum(w * r * q) * q
        rows.append(r / np.sqrt(np.sum(w * r * r)))
    return np.array(rows)


def _make(name, V, W, ghosts):
    v = np.array(V, dtype=np.float64)
    w = np.array(W, dtype=np.float64)
    return _lat.Lattice(name, v=v, w=w, m=basis(v, w, _hydro(v) + ghosts(v)), conserved=(0, 1, 2, 3))


LATTICES = {"D3Q15": _make("D3Q15", V15, W15, _ghosts15), "D3Q19": _make("D3Q19", V19, W19, _ghosts19)}


def lattice_of(q_or_name):
    """The lattice by name or by its number of velocities."""
    if isinstance(q_or_name, str):
        return LATTICES[q_or_name]
    return next(L for L in LATTICES.values() if L.q == q_or_name)


@dataclass
class Params3:
    nx: int = 8
    ny: int = 8
    nz: int = 8
    tau: Sequence[float] = None                # per moment; conserved entries unused; None = all 1
    rho0: float = 1.0
    kT: float = 1.0 / 3.0
    u0: Sequence[float] = (0.0, 0.0, 0.0)
    seed: int = 0
    stream: int = 0
    noise_mask: int = None                     # bit a = noise on moment a; None = all non-conserved
    init_mode: int = 0
    fields: Sequence[int] = field(default_factory=list)
    lattice: str = "D3Q15"

    @property
    def lat(self):
        return LATTICES[self.lattice]

    @property
    def mu(self):
        return 3.0 * self.kT

    def taus(self):
        return np.ones(self.lat.q) if self.tau is None else np.asarray(self.tau, float)

    def mask(self):
        if self.noise_mask is None:
            return sum(1 << a for a in self.lat.nonconserved)
        return int(self.noise_mask)


def site_index(p):
    z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    return ((z * p.ny + y) * p.nx + x).astype(np.uint64)


def uniform_state(p):
    rho = np.full((p.nz, p.ny, p.nx), p.rho0)
    u = np.broadcast_to(np.asarray(p.u0, float)[:, None, None, None], (3, p.nz, p.ny, p.nx))
    return _lat.equilibrium(p.lat, rho, u)


def thermal_state(p):
    """f^0(rho0, u0) plus moment fluctuations N(0, mu rho0) (tag 1), lattice means of the
    density and momentum fluctuations removed."""
    lat = p.lat
    N = _rng.site_normals(lat.q, site_index(p), 0, 1, p.stream, p.seed)
    dM = np.sqrt(p.mu * p.rho0) * N
    for a in lat.conserved:
        dM[a] -= dM[a].mean()
    return uniform_state(p) + np.tensordot(lat.n, dM, axes=(1, 0))


def stream(fstar):
    lat = lattice_of(fstar.shape[0])
    out = np.empty_like(fstar)
    for i, (vx, vy, vz) in enumerate(lat.v.astype(int)):
        out[i] = np.roll(fstar[i], shift=(vz, vy, vx), axis=(0, 1, 2))
    return out


def macroscopic(f):
    lat = lattice_of(f.shape[0])
    rho = f.sum(axis=0)
    j = np.tensordot(lat.v.T, f, axes=(1, 0))
    return rho, j, j / rho


def collide(p, f, t, return_parts=False):
    """Eq. 5 with the noise of Eq. 8 on the masked non-conserved moments."""
    lat = p.lat
    rho, j, u = macroscopic(f)
    M = np.tensordot(lat.m, f, axes=(1, 0))
    Meq = np.tensordot(lat.m, _lat.equilibrium(lat, rho, u), axes=(1, 0))
    tau = p.taus()
    xi = np.zeros_like(M)
    mask = p.mask()
    if any((mask >> a) & 1 for a in lat.nonconserved):
        N = _rng.site_normals(len(lat.nonconserved), site_index(p), t, 0, p.stream, p.seed)
        for c, a in enumerate(lat.nonconserved):
            if (mask >> a) & 1:
                xi[a] = np.sqrt(p.mu * p.rho0 * (2.0 * tau[a] - 1.0)) / tau[a] * N[c]   # Eq. 8
    Mp = M.copy()
    for a in lat.nonconserved:
        Mp[a] = M[a] - (M[a] - Meq[a]) / tau[a] + xi[a]
    fstar = np.tensordot(lat.n, Mp, axes=(1, 0))
    return (fstar, dict(M=M, Meq=Meq, xi=xi, rho=rho, u=u)) if return_parts else fstar


def sample_fields(p, f):
    lat = p.lat
    M = np.tensordot(lat.m, f, axes=(1, 0))
    Mref = lat.m @ _lat.equilibrium(lat, np.array(p.rho0), np.asarray(p.u0, float))
    return {a: M[a] - Mref[a] for a in p.fields}


def dft_at(x, k):
    """X(k) = sum_x X(x) exp(-i k.x) at k = 2 pi (kx/nx, ky/ny, kz/nz), k given as (kz, ky, kx)."""
    nz, ny, nx = x.shape
    kz, ky, kx = k
    ex = np.exp(-2j * np.pi * kx * np.arange(nx) / nx)
    ey = np.exp(-2j * np.pi * ky * np.arange(ny) / ny)
    ez = np.exp(-2j * np.pi * kz * np.arange(nz) / nz)
    return np.einsum("zyx,z,y,x->", x.astype(np.complex128), ez, ey, ex)


class PointAccumulator3:
    """Equal-time C_ab(k) = <X_a(k) X_b(k)^*> / (V mu rho0) at chosen k (no k = 0)."""

    def __init__(self, p, kpoints):
        self.p, self.k = p, [tuple(k) for k in kpoints]
        self.n = 0
        self.sum = {(a, b): np.zeros(len(self.k), complex) for a in p.fields for b in p.fields}

    def add(self, fields):
        X = {a: np.array([dft_at(v, k) for k in self.k]) for a, v in fields.items()}
        for (a, b), s in self.sum.items():
            s += X[a] * np.conj(X[b])
        self.n += 1

    def correlator(self, a, b):
        p = self.p
        return self.sum[(a, b)] / self.n / (p.nx * p.ny * p.nz * p.mu * p.rho0)


class Run3:
    def __init__(self, p, kpoints=()):
        self.p = p
        self.f = thermal_state(p) if p.init_mode == 1 else uniform_state(p)
        self.t = 0
        self.acc = PointAccumulator3(p, kpoints) if (p.fields and len(kpoints)) else None

    def run(self, n, sample_every=0):
        for _ in range(int(n)):
            f = stream(self.f)
            if sample_every and self.acc is not None and self.t % sample_every == 0:
                self.acc.add(sample_fields(self.p, f))
            self.f = collide(self.p, f, self.t)
            self.t += 1
        return self

    def conserved(self):
        rho, j, _ = macroscopic(self.f)
        return np.array([rho.sum(), *j.reshape(3, -1).sum(axis=1)])


def point_theory(p, fields, kpoints):
    """Linear-theory C_ab(k) at the chosen k: discrete Lyapunov equation of the one-step
    operator A_k = P_k J (oracle.theory, written for three dimensions).  NaN where A_k has an
    eigenvalue on the unit circle (k = 0, or a component k_a = pi, where a momentum
    component only flips sign every step and gets no noise)."""
    import scipy.linalg as sla
    from . import theory as _th
    lat = p.lat
    tau = p.taus()
    J = _th.collision_jacobian(lat, tau, p.rho0, np.asarray(p.u0, float))
    sig2 = _th.noise_variances(lat, tau, p.rho0, p.kT, p.mask())
    Qf = lat.n @ np.diag(sig2) @ lat.n.T
    L = lat.m[list(fields)]
    out = {(a, b): np.zeros(len(kpoints), complex) for a in fields for b in fields}
    for j, (kz, ky, kx) in enumerate(kpoints):
        kvec = 2 * np.pi * np.array([kx / p.nx, ky / p.ny, kz / p.nz])
        P = np.exp(-1j * (lat.v @ kvec))
        A = P[:, None] * J
        if np.abs(np.linalg.eigvals(A)).max() > 1.0 - 1e-9:       # k = 0 or a neutral mode (k_a = pi)
            for key in out:
                out[key][j] = np.nan
            continue
        Q = (P[:, None] * Qf) * np.conj(P)[None, :]
        C = sla.solve_discrete_lyapunov(A, Q)
        G = L @ C @ L.conj().T / (p.mu * p.rho0)
        for ia, a in enumerate(fields):
            for ib, b in enumerate(fields):
                out[(a, b)][j] = G[ia, ib]
    return out
