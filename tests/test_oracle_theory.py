"""Pins of the oracle's linear theory against Eq. 7 and the paper's Sec. 3 statements (CPU only)."""
import json
import os

import numpy as np
import pytest

from oracle import lb, spectra, theory
from paper_1010_1233_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.json")))

HYDRO = [0, 9, 10]
LADD = (1 << 3) | (1 << 4) | (1 << 5)


def _params(**kw):
    d = W.replica(**kw)
    d.pop("fields")
    return lb.Params(**d)


@pytest.mark.parametrize("taus", [(1.0, 1.0, 1.0), (0.6, 0.8, 1.3), (0.9, 0.55, 1.7)])
def test_ideal_gas_moments_decouple_for_every_k(taus):
    # Eq. 7: at u0 = 0 with noise on all non-conserved moments <dM^a dM^b> = mu rho0 delta^ab
    p = _params(nx=8, ny=6, tau=W.taus_d2q9(*taus), kT=1e-3)
    fields = list(range(9)) + [9, 10]
    S, ex = theory.theory_spectra(p, fields)
    for (a, b), s in S.items():
        want = 1.0 if a == b else 0.0
        if {a, b} & {9} and {a, b} & {1}:
            want = 1.0          # u_x is momentum / sqrt(3 rho0 kT) units: same field as M^1
        if {a, b} & {10} and {a, b} & {2}:
            want = 1.0
        assert np.abs(s - want)[~ex].max() < 1e-11, (a, b)


def test_d1q3_ideal_gas():
    p = _params(lattice="D1Q3", nx=32, ny=1, tau=W.taus_d1q3(0.8), kT=1e-4)
    S, ex = theory.theory_spectra(p, [0, 1, 2])
    for (a, b), s in S.items():
        assert np.abs(s - (a == b))[~ex].max() < 1e-12
    # only k = 0 (conserved) and k = pi (momentum flips sign every step) are neutral
    assert list(np.flatnonzero(ex[0])) == [0, 16]


def test_ladd_scheme_exact_on_axes_and_wrong_off_axes():
    # Sec. 3 (Figs. 1-3, tau = 1, V = 20^2): without ghost noise S(rho) and S(u_x) are exact
    # on the k_x = 0 and k_y = 0 axes, deviate strongly elsewhere, and the u_x u_y cross
    # correlator reaches about 0.25
    p = _params(nx=20, ny=20, tau=W.taus_d2q9(1.0), kT=1.0 / 3.0, noise_mask=LADD)
    S, ex = theory.theory_spectra(p, HYDRO)
    ok = ~ex
    axes = np.zeros_like(ex)
    axes[0, :] = axes[:, 0] = True
    assert np.abs(S[(0, 0)] - 1)[axes & ok].max() < 1e-12
    assert np.abs(S[(9, 9)][0, :] - 1)[ok[0, :]].max() < 1e-12     # S(u_x) white along k_x
    assert np.abs(S[(0, 0)] - 1)[ok & ~axes].max() > 0.3
    r = np.abs(S[(9, 10)])[ok].max()
    lo, hi = GOLDEN["ladd_max_cross_uxuy"]["band"]
    assert lo < r < hi


def test_ghost_noise_removes_cross_correlators():
    # Abstract / Sec. 3: with ghost noise the cross correlators fall below 0.5 % (the linear
    # theory gives zero up to the finite-difference Jacobian)
    p = _params(nx=20, ny=20, tau=W.taus_d2q9(1.0), kT=1.0 / 3.0)
    S, ex = theory.theory_spectra(p, HYDRO)
    r = max(np.abs(S[k])[~ex].max() for k in S if k[0] != k[1])
    assert r < GOLDEN["ghost_noise_max_cross"]["value"]


def test_galilean_violation_grows_with_mean_velocity():
    # Sec. 3 / Fig. 4: at u_x = 0.1 the moments no longer decouple; the error grows with u0
    devs = []
    u1 = GOLDEN["galilean_violation_velocity"]["value"]
    for u in (0.0, u1, 2 * u1):
        p = _params(nx=12, ny=12, tau=W.taus_d2q9(1.0), kT=1e-4, u0=(u, 0.0))
        S, ex = theory.theory_spectra(p, HYDRO)
        devs.append(max(np.abs(S[k] - (k[0] == k[1]))[~ex].max() for k in S))
    assert devs[0] < 1e-11 and 1e-3 < devs[1] < devs[2]


def test_linear_stability_radius():
    # sweep corner: u0 = 0.3 with tau_shear = 0.55 is linearly unstable, u0 = 0 is not
    bad = _params(nx=16, ny=16, tau=W.taus_d2q9(0.55, 0.55, 1.0), u0=(0.3, 0.0))
    good = _params(nx=16, ny=16, tau=W.taus_d2q9(0.55, 0.55, 1.0), u0=(0.0, 0.0))
    assert theory.spectral_radius(bad) > 1.01
    assert theory.spectral_radius(good) < 1.0 + 1e-12


def test_field_rows_velocity_linearisation():
    # du = (dj - u0 drho) / rho0 against a finite difference of u = j / rho
    p = _params(u0=(0.1, -0.05), rho0=1.2)
    lat = p.lat
    f = lb.uniform_state(p)[:, 0, 0]
    rng = np.random.default_rng(0)
    df = 1e-7 * rng.standard_normal(9)
    u1 = (lat.v.T @ (f + df)) / (f + df).sum()
    u0 = (lat.v.T @ f) / f.sum()
    rows = theory.field_rows(p, [9, 10])
    assert np.abs((u1 - u0) - rows @ df).max() < 1e-12
