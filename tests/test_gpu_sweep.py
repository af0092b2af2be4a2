"""The Galilean-invariance sweep's own replica shapes in one batched launch (GPU).

Eight of the 64 sweep replicas (edges 64, 128, 256, 512; u0_x 0 .. 0.30; tau_shear
0.55 .. 1.0; thermal start; rho, u_x, u_y sampled every 10 steps) run together in
the launch configuration the autotuner picks, and each is compared with the FP64
oracle run of that replica alone: populations after 12 steps and the correlators of
its two samples, element by element.
"""
import numpy as np
import pytest

from oracle import lb, spectra
from paper_1010_1233_gb300 import Sim, workloads as W

pytestmark = pytest.mark.gpu

PICK = (0, 5, 10, 15, 60, 61, 62, 63)


def test_sweep_replicas_batched_match_oracle():
    reps = [W.sweep64()["replicas"][r] for r in PICK]
    assert sorted({p["nx"] for p in reps}) == [64, 128, 256, 512]
    assert max(p["u0"][0] for p in reps) == pytest.approx(0.30)
    sim = Sim(reps, precision="fp32")
    sim.autotune(2)
    sim.run(12, 10)
    for i, p in enumerate(reps):
        ref = lb.Run(lb.Params(**p))
        ref.run(12, 10)
        feq = lb.uniform_state(ref.p)
        err = np.abs(sim.populations(i) - ref.f).max() / np.abs(ref.f - feq).max()
        assert err < 2e-5, (PICK[i], err)
        for a, b in spectra.pairs(p["fields"]):
            o = ref.acc.correlator(a, b)
            g = sim.correlator(i, a, b)
            assert np.abs(g - o).max() < 2e-4 * max(1.0, np.abs(o).max()), (PICK[i], a, b)
