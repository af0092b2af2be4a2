"""Seeded synthetic workloads shared by the CUDA path's tests, the bench and the oracle.

This module holds parameters and random numbers only: no step of the lattice
Boltzmann method, no table of the lattice and no formula of the correlators.
Both the CUDA library and the CPU oracle take what it returns as inputs.

The named workloads are the paper's setting (periodic ideal gas, rho0 = 1,
Sec. 3) at the sizes the library is measured on:

* ``d1q3_L64``     D1Q3, L = 64, FP64, tau = 0.8, kT = 1e-4, u0 = 0, seed 1;
                   1e4 warm-up + 1e5 steps, density/momentum spectra every step.
* ``d2q9_256``     D2Q9 256 x 256, tau_shear = tau_bulk = 0.8, tau_ghost = 1.0,
                   kT = 1e-4, u0 = 0, seed 7, thermal start + 1e4 warm-up,
                   2e5 steps, all nine moment fields every 10 steps.
* ``sweep64``      64 D2Q9 replicas r = 0..63: size {64,128,256,512}[r mod 4],
                   u0_x = 0.02 floor(r / 4), tau_shear = tau_bulk =
                   0.55 + 0.45 ((29 r) mod 64) / 63, tau_ghost = 1, seed r,
                   FP32 storage, 1e4 warm-up, 1e5 steps, sampling every 10.
* ``train16``      16 D2Q9 replicas at 128 x 128 with u0_x = 0.02 i (i = 0..15),
                   taus as ``d2q9_256``; held-out evaluation at u0_x in
                   {0.07, 0.17, 0.27}.
* ``d2q9_16384``   D2Q9 16384 x 16384 FP32 deviation storage, tau_shear =
                   tau_bulk = 0.6, tau_ghost = 1.0, u0 = (0.1, 0.05), kT = 1e-4,
                   noise-scale network on, 1e4 steps, rho/u_x/u_y spectra every 20.
* ``d3q15_512``, ``d3q19_512``  the 3D lattices at 512^3, FP32 deviation storage,
                   tau_shear = tau_bulk = 0.8, tau_ghost = 1.0, u0 = (0.05, 0.02, 0),
                   thermal start, three moment fields every 20 steps into time
                   correlators at 16 wave vectors.
"""
import numpy as np

D1Q3, D2Q9 = "D1Q3", "D2Q9"
FIELD_UX, FIELD_UY = 9, 10


def taus_d2q9(tau_shear, tau_bulk=None, tau_ghost=1.0):
    """Relaxation time per D2Q9 moment (0..8); the conserved entries 0..2 are unused."""
    tb = tau_shear if tau_bulk is None else tau_bulk
    return [1.0, 1.0, 1.0, tau_shear, tau_shear, tb, tau_ghost, tau_ghost, tau_ghost]


def taus_d1q3(tau):
    return [1.0, 1.0, tau] + [1.0] * 6


def replica(lattice=D2Q9, nx=16, ny=16, tau=None, rho0=1.0, kT=1e-4, u0=(0.0, 0.0),
            seed=0, stream=0, noise_mask=None, init_mode=0, fields=(), noise_mode=0):
    """One replica's parameters as a plain dict (keys shared by both sides).

    noise_mode 0: independent noise per non-conserved moment (Eq. 8); 1: correlated
    noise for the mean velocity u0; 2: Eq. 8 with the local density."""
    if tau is None:
        tau = taus_d2q9(1.0) if lattice == D2Q9 else taus_d1q3(1.0)
    return dict(lattice=lattice, nx=int(nx), ny=int(ny if lattice == D2Q9 else 1),
                tau=[float(t) for t in tau], rho0=float(rho0), kT=float(kT),
                u0=(float(u0[0]), float(u0[1])), seed=int(seed), stream=int(stream),
                noise_mask=noise_mask, init_mode=int(init_mode), fields=list(fields),
                noise_mode=int(noise_mode))


D3Q15 = "D3Q15"


def taus_d3q15(tau_shear, tau_bulk=None, tau_ghost=1.0):
    """Relaxation time per D3Q15 moment (0..14): shear 4..8, bulk 9, ghosts 10..14."""
    tb = tau_shear if tau_bulk is None else tau_bulk
    return [1.0] * 4 + [tau_shear] * 5 + [tb] + [tau_ghost] * 5


D3Q19 = "D3Q19"


def taus_d3q19(tau_shear, tau_bulk=None, tau_ghost=1.0):
    """Relaxation time per D3Q19 moment (0..18): shear 4..8, bulk 9, ghosts 10..18."""
    tb = tau_shear if tau_bulk is None else tau_bulk
    return [1.0] * 4 + [tau_shear] * 5 + [tb] + [tau_ghost] * 9


def replica3(nx=8, ny=8, nz=8, tau=None, rho0=1.0, kT=1e-4, u0=(0.0, 0.0, 0.0), seed=0, stream=0,
             noise_mask=None, init_mode=0, fields=(), lattice=D3Q15):
    """One D3Q15 or D3Q19 replica's parameters (keys shared by both sides)."""
    if tau is None:
        tau = taus_d3q15(1.0) if lattice == D3Q15 else taus_d3q19(1.0)
    return dict(lattice=lattice, nx=int(nx), ny=int(ny), nz=int(nz), tau=[float(t) for t in tau],
                rho0=float(rho0), kT=float(kT), u0=tuple(float(v) for v in u0), seed=int(seed),
                stream=int(stream), noise_mask=noise_mask, init_mode=int(init_mode), fields=list(fields),
                noise_mode=0)


def d1q3_L64():
    return dict(replicas=[replica(D1Q3, 64, 1, taus_d1q3(0.8), kT=1e-4, seed=1,
                                  fields=(0, 1))],
                warmup=10_000, steps=100_000, sample_every=1)


def d2q9_256():
    return dict(replicas=[replica(D2Q9, 256, 256, taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, seed=7,
                                  init_mode=1, fields=tuple(range(9)))],
                warmup=10_000, steps=200_000, sample_every=10)


def sweep64():
    reps = []
    for r in range(64):
        L = (64, 128, 256, 512)[r % 4]
        ts = 0.55 + 0.45 * ((29 * r) % 64) / 63.0
        reps.append(replica(D2Q9, L, L, taus_d2q9(ts, ts, 1.0), kT=1e-4,
                            u0=(0.02 * (r // 4), 0.0), seed=r, stream=r, init_mode=1,
                            fields=(0, FIELD_UX, FIELD_UY)))
    return dict(replicas=reps, warmup=10_000, steps=100_000, sample_every=10)


def train16():
    reps = [replica(D2Q9, 128, 128, taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, u0=(0.02 * i, 0.0),
                    seed=100 + i, stream=i, init_mode=1, fields=(0, FIELD_UX, FIELD_UY))
            for i in range(16)]
    return dict(replicas=reps, warmup=10_000, steps=100_000, sample_every=10,
                heldout_u0=(0.07, 0.17, 0.27))


def d2q9_16384(n=16384):
    return dict(replicas=[replica(D2Q9, n, n, taus_d2q9(0.6, 0.6, 1.0), kT=1e-4,
                                  u0=(0.1, 0.05), seed=11, init_mode=0,
                                  fields=(0, FIELD_UX, FIELD_UY))],
                warmup=3, steps=10_000, sample_every=20, mlp=True)


def kpoints3(n, count=16):
    """Wave vectors (kz, ky, kx) of the 3D correlator workloads: the first axis and
    diagonal modes of an n^3 box (none at k = 0 or with a component at pi)."""
    ks = []
    for m in range(1, count + 1):
        k = (m - 1) // 4 + 1
        ks.append([(0, 0, k), (0, k, 0), (k, 0, 0), (k, k, k)][(m - 1) % 4])
    return [tuple(c % n for c in k) for k in ks]


def d3q15_512(n=512):
    """D3Q15 n^3 FP32 deviation storage, tau_shear = tau_bulk = 0.8, tau_ghost = 1.0,
    u0 = (0.05, 0.02, 0), kT = 1e-4, thermal start; density, shear M^4 and bulk M^9
    fields every 20 steps into time correlators (8 lags) at 16 wave vectors."""
    return dict(replicas=[replica3(n, n, n, taus_d3q15(0.8, 0.8, 1.0), kT=1e-4, u0=(0.05, 0.02, 0.0), seed=21,
                                   init_mode=1, fields=(0, 4, 9), lattice=D3Q15)],
                kpoints=kpoints3(n), n_lags=8, sample_every=20)


def d3q19_512(n=512):
    """As d3q15_512 on D3Q19."""
    return dict(replicas=[replica3(n, n, n, taus_d3q19(0.8, 0.8, 1.0), kT=1e-4, u0=(0.05, 0.02, 0.0), seed=21,
                                   init_mode=1, fields=(0, 4, 9), lattice=D3Q19)],
                kpoints=kpoints3(n), n_lags=8, sample_every=20)


def random_perturbation(shape, seed, amp=1.0):
    """Gaussian random numbers of a given shape (e.g. a population perturbation)."""
    return amp * np.random.default_rng(seed).standard_normal(shape)


def mlp_weights(seed, hidden=32, scale=1.0, out_scale=0.1):
    """Random FP32 weights of the 3 -> hidden -> hidden -> 6 noise-scale network."""
    g = np.random.default_rng(seed)
    def lin(n_out, n_in, s):
        return ((s / np.sqrt(n_in)) * g.standard_normal((n_out, n_in))).astype(np.float32)
    return dict(W1=lin(hidden, 3, scale * 8.0), b1=(0.1 * g.standard_normal(hidden)).astype(np.float32),
                W2=lin(hidden, hidden, scale), b2=(0.1 * g.standard_normal(hidden)).astype(np.float32),
                W3=lin(6, hidden, out_scale), b3=(0.01 * g.standard_normal(6)).astype(np.float32))


def mlp_inputs(n, seed, u_scale=0.3, rho_scale=0.02):
    """Random per-site features (u_x, u_y, rho - rho0) for network tests."""
    g = np.random.default_rng(seed)
    return np.stack([u_scale * g.uniform(-1, 1, n), u_scale * g.uniform(-1, 1, n),
                     rho_scale * g.standard_normal(n)], axis=1)


def correlator_tables(R, K, seed, n_pairs=6, n_channels=6):
    """Synthetic S^plain (R, P, K) and responses G (R, C, P, K), complex, for loss tests."""
    g = np.random.default_rng(seed)
    Sp = (1.0 + 0.2 * g.standard_normal((R, n_pairs, K))
          + 0.05j * g.standard_normal((R, n_pairs, K)))
    G = (0.2 * g.standard_normal((R, n_channels, n_pairs, K))
         + 0.02j * g.standard_normal((R, n_channels, n_pairs, K)))
    return Sp, G
