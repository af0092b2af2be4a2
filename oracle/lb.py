"""The fluctuating lattice Boltzmann step of the oracle (test infrastructure only).

One step with index t, written densely in f-space so that it shares no
structure with the CUDA kernels (which use closed-form sparse transforms):

1. Pull-stream (Eq. 1, the streaming half): f_i(x, t) = f*_i(x - v_i, t - 1),
   periodic.  The stored state between steps is the post-collision f*.
2. Density and momentum rho = sum_i f_i, j = sum_i f_i v_i, u = j / rho (Sec. 2).
3. Moments M^a = sum_i m_i^a f_i (Eq. 3), dense with the matrix of Eq. 9.
4. Equilibrium moments M^{a,0} = sum_i m_i^a f_i^0(rho, u) with f^0 from Eq. 2
   (the dense sum; the closed forms of Eq. 10 are a test of it).
5. Collision with noise (Eq. 5): M'^a = M^a - (M^a - M^{a,0}) / tau^a + xi^a.
   xi^a = s_a (1/tau^a) sqrt(mu rho0 (2 tau^a - 1)) N^a (Eq. 8) on every
   non-conserved moment whose bit is set in the noise mask (Sec. 2: stress and
   ghost moments; clearing the ghost bits gives the Ladd scheme of Sec. 3),
   xi^a = 0 on density and momentum (Sec. 2, noise conservation).
6. Back transform f*_i = sum_a n_i^a M'^a with n_i^a = w_i m_i^a (Sec. 2).

Readings where the paper is silent or unit-specific:
* Temperature: Eq. 8 is written in units with k_B T = c_s^2 = 1/3.  With a
  general k_B T the equal-time moment covariance of Eq. 7 is mu rho0 delta^ab
  with mu = 3 k_B T, so the amplitude becomes (1/tau) sqrt(mu rho0 (2 tau - 1)).
* rho-bar in Eq. 8 is the fixed mean density rho0 (noise_mode 2: the site's own
  density rho(x), the local form of the amplitude).
* Fields are sampled on the pre-collision state of step t (after streaming).
* s_a = 1 unless a per-site noise-scale network is given (learned extension,
  not in the paper): s_a = 1 + o_a(u_x, u_y, rho - rho0), see ``oracle.mlp``.
* noise_mode = 1 (extension the paper points to after Eq. 7): the noise on the
  non-conserved moments is correlated, xi = s * (R N) with R from
  ``oracle.correlated`` (Eq. 6 with the covariance of Eq. 7 at f^0(rho0, u0)).

Normals come from ``oracle.philox``: D2Q9 uses the six normals of
``pair_normals`` (sites 2q, 2q + 1 share the counter (q, t, call, stream), calls
0..2) for moments 3..8; D1Q3 normal 0 of ``site_normals`` (counter (site, t,
call | tag << 8, stream)) for moment 2.

Parity: pinned (conservation, shear-wave decay against the continuum viscosity
and the exact linear eigenvalue, uniform-equilibrium fixed point, equal-time
statistics against the linear theory of ``oracle.theory``).
"""
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from . import correlated as _corr
from . import lattice as _lat
from . import philox as _rng
from . import spectra as _spec

FIELD_UX = 9
FIELD_UY = 10


@dataclass
class Params:
    lattice: str = "D2Q9"
    nx: int = 16
    ny: int = 16
    tau: Sequence[float] = (1.0,) * 9       # per moment; conserved entries unused
    rho0: float = 1.0
    kT: float = 1.0 / 3.0
    u0: Sequence[float] = (0.0, 0.0)
    seed: int = 0
    stream: int = 0
    noise_mask: Optional[int] = None         # bit a = noise on moment a; None = all non-conserved
    init_mode: int = 0                       # 0 = uniform f^0(rho0, u0); 1 = thermal
    fields: Sequence[int] = field(default_factory=list)
    mlp: Optional[dict] = None               # {"W1","b1","W2","b2","W3","b3"} FP64 arrays
    mlp_bf16: bool = False                   # round network operands to bfloat16 (tensor-core precision)
    noise_mode: int = 0                      # 0: Eq. 8; 1: correlated (oracle.correlated); 2: Eq. 8 with the local rho

    @property
    def lat(self):
        return _lat.LATTICES[self.lattice]

    @property
    def mu(self):
        return 3.0 * self.kT

    def mask(self):
        lat = self.lat
        if self.noise_mask is None:
            return sum(1 << a for a in lat.nonconserved)
        return int(self.noise_mask)

    def u0_vec(self):
        return np.asarray(self.u0, dtype=np.float64)[: self.lat.d]


def _shape(p):
    return (p.ny, p.nx) if p.lat.d == 2 else (1, p.nx)


def site_index(p):
    ny, nx = _shape(p)
    return (np.arange(ny, dtype=np.uint64)[:, None] * np.uint64(nx)
            + np.arange(nx, dtype=np.uint64)[None, :])


def macroscopic(lat, f):
    rho = f.sum(axis=0)
    j = np.tensordot(lat.v.T, f, axes=(1, 0))               # (d,) + S
    return rho, j, j / rho


def uniform_state(p):
    """Uniform equilibrium f^0(rho0, u0) on every site, shape (q, ny, nx)."""
    lat = p.lat
    ny, nx = _shape(p)
    rho = np.full((ny, nx), p.rho0)
    u = np.broadcast_to(p.u0_vec()[:, None, None], (lat.d, ny, nx))
    return _lat.equilibrium(lat, rho, u)


def thermal_state(p):
    """Equilibrium f^0(rho0, u0) plus independent moment fluctuations.

    dM^a ~ N(0, mu rho0) for every moment a and site (generator tag 1, step 0);
    the site average of the density and momentum fluctuations is removed so
    that total mass and momentum equal those of the uniform state exactly.  At
    u0 = 0 this is the stationary law of the linearised dynamics (Eq. 7).
    """
    lat = p.lat
    N = _rng.site_normals(lat.q, site_index(p), 0, 1, p.stream, p.seed)    # (q, ny, nx)
    dM = np.sqrt(p.mu * p.rho0) * N
    for a in lat.conserved:
        dM[a] -= dM[a].mean()
    return uniform_state(p) + np.tensordot(lat.n, dM, axes=(1, 0))


def initial_state(p):
    return thermal_state(p) if p.init_mode == 1 else uniform_state(p)


def stream(lat, fstar):
    """Pull streaming f_i(x) = f*_i(x - v_i) on the periodic lattice."""
    out = np.empty_like(fstar)
    for i in range(lat.q):
        vx = int(lat.v[i, 0])
        vy = int(lat.v[i, 1]) if lat.d == 2 else 0
        out[i] = np.roll(fstar[i], shift=(vy, vx), axis=(0, 1))
    return out


def noise_scale(p, rho, u):
    """Per-site multipliers s_a of the noise amplitudes, array (q,) + S."""
    lat = p.lat
    s = np.ones((lat.q,) + rho.shape)
    if p.mlp is not None:
        from . import mlp as _mlp
        feats = np.stack([u[0], u[1], rho - p.rho0], axis=-1).reshape(-1, 3)
        out = _mlp.forward(p.mlp, feats, bf16_operands=p.mlp_bf16)["s"]     # (sites, 6)
        for c, a in enumerate(lat.nonconserved):
            s[a] = out[:, c].reshape(rho.shape)
    return s


def sample_fields(p, f, rho, u):
    """Fields of the pre-collision state, minus their reference-state values.

    Field id a < q: moment M^a - M^{a,0}(rho0, u0); id 9: u_x - u0_x; id 10: u_y - u0_y.
    Subtracting a constant only changes k = 0, where the sampled mean is removed.
    """
    lat = p.lat
    out = {}
    M = np.tensordot(lat.m, f, axes=(1, 0))
    Mref = lat.m @ _lat.equilibrium(lat, np.array(p.rho0), p.u0_vec())
    u0 = p.u0_vec()
    for fid in p.fields:
        if fid < lat.q:
            out[fid] = M[fid] - Mref[fid]
        elif fid == FIELD_UX:
            out[fid] = u[0] - u0[0]
        elif fid == FIELD_UY:
            out[fid] = u[1] - u0[1]
        else:
            raise ValueError(f"unknown field id {fid}")
    return out


def collide(p, f, t, return_parts=False, sites=None):
    """Collision with noise (Eq. 5) at step t on the pre-collision state f.

    sites: global site indices y*nx + x of the entries of f (default: the whole
    lattice of p); lets a patch of a large lattice be collided on its own.
    """
    lat = p.lat
    if sites is None:
        sites = site_index(p)
    rho, j, u = macroscopic(lat, f)
    M = np.tensordot(lat.m, f, axes=(1, 0))                           # Eq. 3
    Meq = np.tensordot(lat.m, _lat.equilibrium(lat, rho, u), axes=(1, 0))   # Eq. 2 -> moments
    tau = np.asarray(p.tau, dtype=np.float64)
    xi = np.zeros_like(M)
    mask = p.mask()
    active = [a for a in lat.nonconserved if (mask >> a) & 1]
    if active:
        if lat.name == "D2Q9":
            N = _rng.pair_normals(sites, t, 0, p.stream, p.seed)
        else:
            N = _rng.site_normals(1, sites, t, 0, p.stream, p.seed)
        s = noise_scale(p, rho, u)
        if p.noise_mode == 1:                                          # xi = R N (Eqs. 6-7 at u0)
            R, _, _ = _corr.noise_root(lat, tau, p.rho0, p.kT, p.u0_vec(), mask)
            Z = np.tensordot(R, N[: len(lat.nonconserved)], axes=(1, 0))
            for c, a in enumerate(lat.nonconserved):
                xi[a] = s[a] * Z[c]
        else:
            # Eq. 8 with rho-bar = rho0, or with the local density (noise_mode 2)
            rho_n = rho if p.noise_mode == 2 else p.rho0
            for c, a in enumerate(lat.nonconserved):
                if (mask >> a) & 1:
                    amp = np.sqrt(p.mu * rho_n * (2.0 * tau[a] - 1.0)) / tau[a]   # Eq. 8
                    xi[a] = s[a] * amp * N[c]
    Mp = M.copy()
    for a in lat.nonconserved:
        Mp[a] = M[a] - (M[a] - Meq[a]) / tau[a] + xi[a]                # Eq. 5
    fstar = np.tensordot(lat.n, Mp, axes=(1, 0))                      # f*_i = sum_a n_i^a M'^a
    if return_parts:
        return fstar, dict(rho=rho, u=u, M=M, Meq=Meq, xi=xi)
    return fstar


class Run:
    """State (post-collision f*), global step counter and correlator sums; optional
    time correlators at selected wave vectors (``tacc``, spectra.TimeAccumulator)."""

    def __init__(self, p: Params, fstar=None, time_k=None, n_lags=0):
        self.p = p
        self.f = initial_state(p) if fstar is None else np.array(fstar, dtype=np.float64)
        self.t = 0
        self.acc = _spec.Accumulator(p) if p.fields else None
        self.tacc = _spec.TimeAccumulator(p, time_k, n_lags) if (time_k and p.fields) else None

    def run(self, n_steps, sample_every=0):
        p = self.p
        for _ in range(int(n_steps)):
            f = stream(p.lat, self.f)
            if sample_every and self.acc is not None and self.t % sample_every == 0:
                rho, _, u = macroscopic(p.lat, f)
                fl = sample_fields(p, f, rho, u)
                self.acc.add(fl)
                if self.tacc is not None:
                    self.tacc.add(fl)
            self.f = collide(p, f, self.t)
            self.t += 1
        return self

    def conserved(self):
        rho, j, _ = macroscopic(self.p.lat, self.f)
        return np.concatenate([[rho.sum()], j.reshape(j.shape[0], -1).sum(axis=1)])
