"""Validation of flb_replica under random and invalid parameters (CPU only): the library
either sizes a workspace at least as large as the population buffers or returns
FLB_EINVAL with a message; it never crashes."""
import ctypes

import numpy as np

from paper_1010_1233_gb300 import _lib as L


def _valid(g):
    lat = int(g.choice([1, 2, 3, 4]))
    s = L.flb_replica()
    s.lattice = lat
    s.nx = int(g.choice([2, 4, 8, 16, 24, 64]))
    s.ny = 1 if lat == 1 else int(g.choice([1, 2, 3, 8, 16]))
    s.nz = int(g.choice([1, 2, 5])) if lat >= 3 else 1
    for a in range(20):
        s.tau[a] = float(g.uniform(0.55, 2.0))
    s.rho0, s.kT = 1.0, 1e-4
    s.u0[0], s.u0[1], s.u0[2] = 0.05, -0.02, 0.0
    s.seed, s.stream = int(g.integers(0, 2**63)), int(g.integers(0, 2**31))
    s.noise_mask = 0xFFFFFFFF & (((1 << {1: 3, 2: 9, 3: 15, 4: 19}[lat]) - 1) & ~((1 << (2 if lat == 1 else (3 if lat == 2 else 4))) - 1))
    s.init_mode = int(g.integers(0, 2))
    s.field_mask = 0
    s.noise_mode = 0
    return s


MUTATIONS = [
    ("lattice", [0, 5, -1]), ("nx", [0, 1, 3, -2, 1 << 20]), ("ny", [0, -1, 1 << 16]), ("nz", [0, -1, 1 << 12]),
    ("rho0", [0.0, -1.0, float("nan")]), ("kT", [-1e-4, float("inf")]), ("init_mode", [2, 7]),
    ("noise_mode", [1, 2, 3]), ("noise_mask", [1, 1 << 2, 1 << 19, 0xFFFFFFFF]),
    ("field_mask", [1, 0x7, 0x601, 0x7FF, 0x7FFF, 1 << 18, 1 << 31]),
]


def _case(g):
    s = _valid(g)
    for _ in range(int(g.integers(0, 3))):
        name, vals = MUTATIONS[int(g.integers(0, len(MUTATIONS)))]
        setattr(s, name, vals[int(g.integers(0, len(vals)))])
    if g.random() < 0.2:
        s.tau[int(g.integers(0, 20))] = float(g.choice([0.5, 0.3, float("nan"), float("inf")]))
    if g.random() < 0.1:
        s.u0[int(g.integers(0, 3))] = float("nan")
    return s


def test_random_parameters_are_validated():
    lib = L.lib()
    g = np.random.default_rng(123)
    ok = bad = 0
    for _ in range(3000):
        s = _case(g)
        n = ctypes.c_size_t()
        prec = int(g.choice([L.FLB_FP64, L.FLB_FP32_DEV, 7]))
        rc = lib.flb_workspace_bytes(prec, (L.flb_replica * 1)(s), 1, ctypes.byref(n))
        if rc == 0:
            ok += 1
            q = {1: 3, 2: 9, 3: 15, 4: 19}[s.lattice]
            V = s.nx * s.ny * (s.nz if s.lattice >= 3 else 1)
            assert n.value >= 2 * q * V * (8 if prec == L.FLB_FP64 else 4)
        else:
            assert rc == L.FLB_EINVAL, rc
            assert len(lib.flb_last_error()) > 0
            bad += 1
    assert ok > 300 and bad > 300, (ok, bad)
