"""Pins of the oracle's DFT and correlator normalisation (Eqs. 11-12) (CPU only)."""
import numpy as np

from oracle import lb, spectra
from paper_1010_1233_gb300 import workloads as W


def test_dft_matches_library_fft_and_parseval():
    x = W.random_perturbation((6, 10), 3)
    X = spectra.dft2(x)
    assert np.abs(X - np.fft.fft2(x)).max() < 1e-12
    assert abs(np.sum(np.abs(X) ** 2) / x.size - np.sum(x**2)) < 1e-12


def test_dft_single_mode():
    ny, nx, kx, ky = 8, 12, 3, 5
    y, x = np.mgrid[0:ny, 0:nx]
    X = spectra.dft2(np.cos(2 * np.pi * (kx * x / nx + ky * y / ny)))
    want = np.zeros((ny, nx), complex)
    want[ky, kx] = want[-ky, -kx] = nx * ny / 2
    assert np.abs(X - want).max() < 1e-11


def test_white_noise_normalises_to_one():
    # a field of independent sites with the ideal-gas variance mu rho0 has S = 1 at all k != 0
    d = W.replica(nx=8, ny=8, kT=0.02, rho0=1.3, fields=[0, 9])
    p = lb.Params(**d)
    acc = spectra.Accumulator(p)
    rng = np.random.default_rng(0)
    n = 4000
    for _ in range(n):
        acc.add({0: np.sqrt(p.mu * p.rho0) * rng.standard_normal((8, 8)) + 5.0,
                 9: np.sqrt(p.kT / p.rho0) * rng.standard_normal((8, 8)) - 2.0})
    for a, b, want in ((0, 0, 1.0), (9, 9, 1.0), (0, 9, 0.0)):
        C = acc.correlator(a, b)
        # k = 0 included: the sampled mean is subtracted there
        assert np.abs(C - want).max() < 6 / np.sqrt(n)


def test_correlator_hermitian_symmetry():
    d = W.replica(nx=6, ny=4, fields=[0, 9])
    p = lb.Params(**d)
    acc = spectra.Accumulator(p)
    for s in range(5):
        acc.add({0: W.random_perturbation((4, 6), s), 9: W.random_perturbation((4, 6), 10 + s)})
    C = acc.correlator(0, 9)
    Cm = np.roll(np.flip(C, (0, 1)), 1, (0, 1))        # C(-k)
    assert np.abs(C - np.conj(Cm)).max() < 1e-13 * np.abs(C).max()
    assert np.abs(acc.correlator(9, 0) - np.conj(C)).max() < 1e-15


def test_point_accumulator_equals_full_grid():
    d = W.replica(nx=8, ny=4, kT=0.01, fields=[0, 9])
    p = lb.Params(**d)
    ks = [(0, 0), (1, 3), (3, 7), (2, 4)]
    full, pts = spectra.Accumulator(p), spectra.PointAccumulator(p, ks)
    for s in range(4):
        f = {0: W.random_perturbation((4, 8), s) + 1.0, 9: W.random_perturbation((4, 8), 20 + s)}
        full.add(f)
        pts.add(f)
    for a, b in ((0, 0), (0, 9), (9, 9)):
        C = full.correlator(a, b)
        assert np.abs(pts.correlator(a, b) - np.array([C[ky, kx] for ky, kx in ks])).max() < 1e-12
