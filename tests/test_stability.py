"""flb_stability (host-side linear stability pre-check, no GPU) against the oracle's
linear theory: the same one-step operator A_k = P_k J on the same k-grid (CPU only)."""
import itertools

import numpy as np
import pytest

from oracle import lb, lb3d, theory
from paper_1010_1233_gb300 import _lib as L, stability, workloads as W


def _oracle_radius(lat, tau, rho0, u0, dims):
    J = theory.collision_jacobian(lat, np.asarray(tau, float), rho0, np.asarray(u0, float))
    r = 0.0
    for idx in itertools.product(*[range(n) for n in dims]):
        k = np.array([2 * np.pi * j / n for j, n in zip(idx, dims)])
        P = np.exp(-1j * (lat.v @ k))
        r = max(r, np.abs(np.linalg.eigvals(P[:, None] * J)).max())
    return r


CASES2 = [
    (W.taus_d2q9(0.8, 0.8, 1.0), (0.0, 0.0)),
    (W.taus_d2q9(0.55, 0.55, 1.0), (0.3, 0.0)),          # unstable at large u0 and small tau
    (W.taus_d2q9(0.6, 0.9, 1.4), (0.15, -0.1)),
    (W.taus_d2q9(0.52, 0.52, 0.52), (0.2, 0.2)),
]


@pytest.mark.parametrize("tau,u0", CASES2)
def test_d2q9_matches_oracle(tau, u0):
    p = W.replica("D2Q9", 16, 12, tau, u0=u0)
    r, k = stability(p, max_k=64)
    ro = theory.spectral_radius(lb.Params(**p))
    assert abs(r - ro) < 1e-7 * ro, (r, ro)
    assert r >= 1.0 - 1e-9                                 # k = 0 carries the conserved modes


def test_known_unstable_and_stable_cases():
    r, _ = stability(W.replica("D2Q9", 64, 64, W.taus_d2q9(0.55, 0.55, 1.0), u0=(0.3, 0.0)))
    assert r > 1.01
    r, _ = stability(W.replica("D2Q9", 64, 64, W.taus_d2q9(0.8, 0.8, 1.0), u0=(0.1, 0.05)))
    assert abs(r - 1.0) < 1e-9


def test_d1q3_matches_oracle():
    for tau, u in ((0.8, 0.0), (0.55, 0.3), (0.6, -0.2)):
        p = W.replica("D1Q3", 32, 1, W.taus_d1q3(tau), u0=(u, 0.0))
        r, _ = stability(p)
        ro = _oracle_radius(lb.Params(**p).lat, p["tau"], 1.0, (u,), (32,))
        assert abs(r - ro) < 1e-7 * ro, (tau, u, r, ro)


@pytest.mark.parametrize("lat", ["D3Q15", "D3Q19"])
def test_3d_matches_oracle(lat):
    tau = W.taus_d3q15(0.6, 0.8, 1.1) if lat == "D3Q15" else W.taus_d3q19(0.6, 0.8, 1.1)
    for u0 in ((0.0, 0.0, 0.0), (0.25, -0.1, 0.15)):
        p = W.replica3(6, 4, 4, tau, u0=u0, lattice=lat)
        r, _ = stability(p, max_k=8)
        ro = _oracle_radius(lb3d.LATTICES[lat], tau, 1.0, u0, (6, 4, 4))
        assert abs(r - ro) < 1e-7 * ro, (lat, u0, r, ro)


def test_invalid_replica_rejected():
    with pytest.raises(L.FlbError):
        stability(W.replica("D2Q9", 16, 16, W.taus_d2q9(0.5)))
    with pytest.raises(L.FlbError):
        stability(W.replica("D2Q9", 16, 16), max_k=0)
