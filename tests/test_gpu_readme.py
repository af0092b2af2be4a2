"""The usage shown in README.md runs as written (fewer steps), 2D and 3D (GPU)."""
import numpy as np
import pytest

from paper_1010_1233_gb300 import Sim, stability, workloads as W

pytestmark = pytest.mark.gpu


def test_readme_2d_example():
    p = W.replica("D2Q9", 256, 256, W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, seed=7, init_mode=1,
                  fields=(0, W.FIELD_UX, W.FIELD_UY))
    sim = Sim(p, precision="fp32")
    vec, grid, staged, ms = sim.autotune(2)
    assert vec in (1, 2, 4) and ms > 0
    sim.run(200)
    sim.reset_stats()
    sim.run(400, sample_every=10)
    S, n = sim.correlator(0, 0, 0, with_count=True)
    assert S.shape == (256, 256) and n == 40
    k = np.ones_like(S.real, dtype=bool)
    k[0, 0] = False
    assert abs(S.real[k].mean() - 1.0) < 0.1           # flat at u0 = 0 (Eq. 7), 40 samples
    c = sim.conserved()
    assert c.shape == (3,) and abs(c[0] - 256 * 256) < 1e-2
    r, _ = stability(p)
    assert abs(r - 1.0) < 1e-9


def test_readme_3d_time_correlators():
    p = W.replica3(32, 32, 32, W.taus_d3q19(0.8), kT=1e-4, seed=3, init_mode=1, fields=(0, 4), lattice="D3Q19")
    sim = Sim(p, precision="fp32")
    sim.set_time_correlator([(0, 0, 1), (1, 2, 3)], 4)
    sim.run(400, sample_every=2)
    F, n = sim.time_correlator(0, 4, 4, with_count=True)
    assert F.shape == (4, 2) and n == 200
    assert abs(F[0].real.mean() - 1.0) < 0.15            # equal-time, flat at u0 = 0
