"""D3Q15 and D3Q19 CUDA paths against the FP64 oracle (oracle.lb3d), through the C ABI (GPU).

The step, the thermal start, the lattice sums and the time correlators at chosen wave
vectors, element by element on the same seeded inputs; then the simulated equal-time
spectra against the linear theory."""
import numpy as np
import pytest

from oracle import lb3d as D
from paper_1010_1233_gb300 import Sim, workloads as W

LATS = ["D3Q15", "D3Q19"]


def _taus(lat, *a):
    return W.taus_d3q15(*a) if lat == "D3Q15" else W.taus_d3q19(*a)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12        # per step, relative to max |f - f^0(rho0, u0)|
FP32_TOL = 2e-5         # after the run, relative to max |f - f^0(rho0, u0)|


def _params(p):
    return D.Params3(nx=p["nx"], ny=p["ny"], nz=p["nz"], tau=p["tau"], rho0=p["rho0"], kT=p["kT"],
                     u0=p["u0"], seed=p["seed"], stream=p["stream"], noise_mask=p["noise_mask"],
                     init_mode=p["init_mode"], fields=list(p["fields"]), lattice=p["lattice"])


def _rel(a, b, ref):
    return np.abs(a - b).max() / max(np.abs(ref).max(), 1e-12)


CASES = [
    (8, 6, 4, dict(taus=(0.8, 0.8, 1.0), init_mode=1)),
    (16, 12, 10, dict(taus=(0.6, 0.9, 1.3), u0=(0.1, -0.05, 0.07), init_mode=1)),   # 7.5 blocks
    (10, 3, 5, dict(taus=(0.7, 0.7, 1.0), u0=(-0.05, 0.1, 0.0), noise_mask=(1 << 5) | (1 << 9) | (1 << 14))),
    (2, 1, 1, dict(taus=(0.9,), init_mode=1)),                                       # degenerate box
]


@pytest.mark.parametrize("lat", LATS)
@pytest.mark.parametrize("nx,ny,nz,kw", CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}" for c in CASES])
def test_fp64_step_matches_oracle_every_step(lat, nx, ny, nz, kw):
    kw = dict(kw)
    kw["tau"] = _taus(lat, *kw.pop("taus"))
    p = W.replica3(nx, ny, nz, kT=1e-3, seed=11, stream=3, lattice=lat, **kw)
    sim = Sim(p, precision="fp64")
    ref = D.Run3(_params(p))
    feq = D.uniform_state(ref.p)
    assert np.abs(sim.populations() - ref.f).max() < 1e-15 * np.abs(ref.f).max()
    worst = 0.0
    for _ in range(30):
        sim.run(1)
        ref.run(1)
        worst = max(worst, _rel(sim.populations(), ref.f, ref.f - feq))
    assert worst < FP64_TOL, worst
    c = sim.conserved()
    assert c.shape == (4,)
    assert np.abs(c - ref.conserved()).max() < 1e-12 * nx * ny * nz


@pytest.mark.parametrize("lat", LATS)
@pytest.mark.parametrize("vec", [1, 2, 4])
def test_fp32_step_matches_oracle(lat, vec):
    p = W.replica3(16, 12, 10, _taus(lat, 0.6, 0.9, 1.3), kT=1e-3, u0=(0.1, -0.05, 0.07), seed=5, stream=1,
                   init_mode=1, lattice=lat)
    sim = Sim(p, precision="fp32")
    sim.set_step_config(vec)
    ref = D.Run3(_params(p))
    feq = D.uniform_state(ref.p)
    sim.run(40)
    ref.run(40)
    assert _rel(sim.populations(), ref.f, ref.f - feq) < FP32_TOL


@pytest.mark.parametrize("lat", LATS)
def test_batched_replicas_and_graphs(lat):
    reps = [W.replica3(8, 6, 4, _taus(lat, 0.8), kT=1e-3, seed=1, init_mode=1, lattice=lat),
            W.replica3(12, 4, 6, _taus(lat, 0.6, 1.1, 1.4), kT=2e-3, u0=(0.05, 0.0, -0.1), seed=2, stream=9,
                       init_mode=1, lattice=lat)]
    sim = Sim(reps, precision="fp64")
    sim.run(70)                                    # graph chunks of 32 steps plus direct steps
    for r, p in enumerate(reps):
        ref = D.Run3(_params(p)).run(70)
        feq = D.uniform_state(ref.p)
        assert _rel(sim.populations(r), ref.f, ref.f - feq) < 1e-11
    plain = Sim(reps, precision="fp64")
    plain.set_graphs(False)
    plain.run(70)
    for r in range(2):
        assert np.array_equal(plain.populations(r), sim.populations(r))


@pytest.mark.parametrize("lat", LATS)
def test_conservation_long_run_fp32(lat):
    p = W.replica3(32, 16, 8, _taus(lat, 0.55, 0.7, 1.0), kT=1e-2, u0=(0.1, 0.05, -0.02), seed=4, init_mode=1,
                   lattice=lat)
    sim = Sim(p, precision="fp32")
    c0 = sim.conserved()
    sim.run(500)
    c1 = sim.conserved()
    V = 32 * 16 * 8
    assert abs(c1[0] - c0[0]) < 1e-4 * V * 1e-2
    assert np.abs(c1[1:] - c0[1:]).max() < 1e-4 * V * 1e-2


@pytest.mark.parametrize("lat", LATS)
def test_checkpoint_roundtrip(lat):
    p = W.replica3(8, 8, 8, _taus(lat, 0.7), kT=1e-3, seed=9, init_mode=1, fields=(0, 4), lattice=lat)
    a = Sim(p, precision="fp32")
    a.run(7)
    blob = a.save()
    a.run(9)
    b = Sim(p, precision="fp32")
    b.load(blob)
    b.run(9)
    assert np.array_equal(a.populations(), b.populations())


def _oracle_series(p, n_steps, every, kpoints):
    """Per sample: {field: X_f(k) for k in kpoints} from the oracle's trajectory."""
    ref = D.Run3(_params(p))
    out = []
    for _ in range(n_steps):
        f = D.stream(ref.f)
        if ref.t % every == 0:
            fl = D.sample_fields(ref.p, f)
            out.append({a: np.array([D.dft_at(v, k) for k in kpoints]) for a, v in fl.items()})
        ref.f = D.collide(ref.p, f, ref.t)
        ref.t += 1
    return out


@pytest.mark.parametrize("lat", LATS)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_time_correlators_match_oracle(lat, precision, tol):
    fields = (0, 2, 5, 9, 13) if lat == "D3Q15" else (0, 3, 9, 13, 16, 18)
    p = W.replica3(12, 8, 6, _taus(lat, 0.7, 0.9, 1.2), kT=1e-3, u0=(0.05, 0.02, -0.03), seed=21, init_mode=1,
                   fields=fields, lattice=lat)
    kpoints = [(0, 0, 1), (0, 1, 0), (1, 0, 0), (2, 3, 5), (5, 7, 11), (3, 4, 6), (1, 1, 1)]
    T, every, n = 4, 2, 24
    sim = Sim(p, precision=precision)
    sim.set_time_correlator(kpoints, T)
    sim.run(n, sample_every=every)
    ser = _oracle_series(p, n, every, kpoints)
    V = 12 * 8 * 6
    norm = V * 3 * p["kT"] * p["rho0"]
    for a in fields:
        for b in fields:
            got, cnt = sim.time_correlator(0, a, b, with_count=True)
            assert cnt == len(ser)
            for tau in range(T):
                want = np.mean([ser[s][a] * np.conj(ser[s - tau][b]) for s in range(tau, len(ser))], axis=0) / norm
                scale = np.abs(want).max() + 1e-30
                assert np.abs(got[tau] - want).max() < tol * max(scale, 1.0), (a, b, tau)


@pytest.mark.parametrize("lat", LATS)
def test_sampled_fields_match_oracle(lat):
    fields = (0, 1, 3, 4, 8, 10, 14) if lat == "D3Q15" else (0, 2, 5, 9, 11, 15, 17, 18)
    p = W.replica3(10, 6, 4, _taus(lat, 0.8), kT=1e-3, u0=(0.02, 0.0, 0.04), seed=2, init_mode=1, fields=fields,
                   lattice=lat)
    sim = Sim(p, precision="fp64")
    sim.set_time_correlator([(0, 0, 1)], 1)
    sim.run(5, sample_every=4)                      # samples at steps 0 and 4
    ref = D.Run3(_params(p))
    ref.run(4)
    want = D.sample_fields(ref.p, D.stream(ref.f))
    got = sim.fields()
    for s, a in enumerate(fields):
        assert np.abs(got[s] - want[a]).max() < 1e-13, a


@pytest.mark.parametrize("lat", LATS)
def test_equal_time_spectra_match_linear_theory(lat):
    # FP32 box of 16^3 sites, thermal start, shear and ghost moments: the simulated C_aa(k)
    # against the discrete Lyapunov solution of the linear theory (flat at u0 = 0)
    fields = (4, 6, 9, 10, 13, 14) if lat == "D3Q15" else (4, 6, 9, 10, 14, 16, 18)
    p = W.replica3(16, 16, 16, _taus(lat, 0.8, 0.8, 1.0), kT=1e-4, seed=33, init_mode=1, fields=fields,
                   lattice=lat)
    kpoints = [(0, 0, 1), (0, 2, 1), (1, 3, 2), (4, 4, 4), (2, 0, 5), (7, 1, 3), (3, 5, 6), (6, 6, 2)]
    sim = Sim(p, precision="fp32")
    sim.run(500)
    sim.set_time_correlator(kpoints, 1)
    sim.run(6000, sample_every=3)
    th = D.point_theory(_params(p), fields, kpoints)
    ratios = []
    for a in fields:
        got = sim.time_correlator(0, a, a)[0].real
        want = th[(a, a)].real
        assert np.all(np.isfinite(want))
        ratios.append(got / want)
    ratios = np.array(ratios)
    # 2000 samples each; relaxation within a few steps, so the relative error of one
    # entry is ~ 1/sqrt(2000 / 2) = 3%; the mean over ~50 entries is good to ~0.5%
    assert np.abs(ratios - 1).max() < 0.15, ratios
    assert abs(ratios.mean() - 1) < 0.02, ratios.mean()
