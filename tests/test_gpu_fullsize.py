"""The CUDA path at the 16384^2 size and in the launch configuration bench.py times (GPU).

The oracle cannot run the whole lattice, so it checks sampled outputs: one step
of a window of the full lattice (from the window plus a one-site halo read back
before the step), and correlators at sampled wave vectors of lattices as long as
16384 in each direction (row transforms of 16384 points, four-step columns).
"""
import numpy as np
import pytest

from oracle import lb, mlp as omlp, spectra
from paper_1010_1233_gb300 import Sim, workloads as W

pytestmark = pytest.mark.gpu


def _window_step(sim, P, x0, y0, w, h):
    before = sim.populations_window(x0 - 1, y0 - 1, w + 2, h + 2)
    t = sim.step
    sim.run(1, 20)
    after = sim.populations_window(x0, y0, w, h)
    f = np.empty((9, h, w))
    for i, (vx, vy) in enumerate(P.lat.v.astype(int)):
        f[i] = before[i, 1 - vy:1 - vy + h, 1 - vx:1 - vx + w]
    sites = ((y0 + np.arange(h, dtype=np.uint64))[:, None] * np.uint64(P.nx)
             + (x0 + np.arange(w, dtype=np.uint64))[None, :])
    fstar = lb.collide(P, f, t, sites=sites)
    feq = lb.uniform_state(lb.Params(**dict(W.d2q9_16384(8)["replicas"][0])))[:, :1, :1]
    return np.abs(after - fstar).max() / np.abs(fstar - feq).max()


@pytest.mark.parametrize("with_mlp,tol", [(False, 2e-5), (True, 1e-3)])
def test_full_lattice_window_step(with_mlp, tol):
    p = W.d2q9_16384()["replicas"][0]
    sim = Sim(p, precision="fp32")
    P = lb.Params(**p)
    if with_mlp:
        wts = W.mlp_weights(1234, out_scale=0.1)
        sim.set_mlp(wts)
        P.mlp = {k: (omlp.to_bf16(v) if k.startswith("W") else v.astype(np.float64)) for k, v in wts.items()}
        P.mlp_bf16 = True
    sim.run(21, 20)                   # two sampling steps included (t = 0, 20)
    errs = [_window_step(sim, P, 5000, 9000, 96, 6), _window_step(sim, P, 16383 - 97, 16383 - 7, 96, 6)]
    assert max(errs) < tol, errs
    c0 = sim.conserved()
    sim.run(20, 20)
    c1 = sim.conserved()
    V = p["nx"] * p["ny"]
    assert abs(c1[0] - c0[0]) < 1e-9 * V and np.abs(c1[1:] - c0[1:]).max() < 1e-9 * V
    sim.close()


@pytest.mark.parametrize("nx,ny", [(16384, 32), (32, 16384)])
def test_long_transforms_at_sampled_wavevectors(nx, ny):
    fields = (0, W.FIELD_UX, W.FIELD_UY)
    p = W.replica("D2Q9", nx, ny, W.taus_d2q9(0.6, 0.6, 1.0), kT=1e-4, u0=(0.1, 0.05), seed=13,
                  init_mode=1, fields=fields)
    sim = Sim(p, precision="fp32")
    rng = np.random.default_rng(0)
    ks = [(0, 0), (0, 1), (1, 0), (ny // 2, nx // 2), (ny - 1, nx - 1)]
    ks += [(int(rng.integers(ny)), int(rng.integers(nx))) for _ in range(15)]
    P = lb.Params(**p)
    ref = lb.Run(P)
    ref.acc = spectra.PointAccumulator(P, ks)
    sim.run(3, 1)
    ref.run(3, 1)
    for a, b in spectra.pairs(fields):
        g = sim.correlator(0, a, b)
        o = ref.acc.correlator(a, b)
        got = np.array([g[ky, kx] for ky, kx in ks])
        err = np.abs(got - o).max() / max(1.0, np.abs(o).max())
        assert err < 2e-4, (a, b, err)
