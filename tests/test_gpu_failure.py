"""Failure detection without a GPU fault (GPU).

A linearly unstable replica (u0 = 0.5, tau = 0.505: spectral radius ~1.46 per step
by the linear theory) blows up to non-finite values within a few hundred steps;
the conservation check must turn that into FLB_EUNSTABLE on the host, and the
status must stay set.  Non-finite values are ordinary IEEE arithmetic on the
device: nothing faults or hangs.  A bounded wait that runs out is reported as
FLB_ETIMEOUT.
"""
import time

import numpy as np
import pytest

from oracle import lb, theory
from paper_1010_1233_gb300 import Sim, workloads as W
from paper_1010_1233_gb300 import _lib as L

pytestmark = pytest.mark.gpu


def test_unstable_replica_reported():
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.505, 0.505, 1.0), kT=1e-3, u0=(0.5, 0.0), seed=1, init_mode=1)
    assert theory.spectral_radius(lb.Params(**p)) > 1.3
    stable = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8), kT=1e-3, seed=2, stream=1, init_mode=1)
    sim = Sim([stable, p], precision="fp32")
    sim.run(2000)
    assert np.all(np.isfinite(sim.conserved(0)))          # the stable replica is fine
    with pytest.raises(L.FlbError) as e:
        sim.conserved(1)
    assert e.value.code == L.FLB_EUNSTABLE
    with pytest.raises(L.FlbError) as e:                   # sticky until the context is rebuilt
        sim.sync()
    assert e.value.code == L.FLB_EUNSTABLE


def test_bounded_wait_timeout_reported():
    """A bounded device wait that nothing completes (the mbarrier wait of the network
    kernels, limited to 2^26 SM clocks) gives up, the host reads FLB_ETIMEOUT, and the
    device stays usable.  The wait is on an mbarrier no thread or copy arrives at: no
    asynchronous operation is in flight, nothing faults or hangs."""
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8), kT=1e-4, seed=1)
    sim = Sim(p, precision="fp32")
    sim.sync()
    with pytest.raises(L.FlbError) as e:
        sim.probe_wait_timeout(0)
    assert e.value.code == L.FLB_EINVAL
    t0 = time.perf_counter()
    sim.probe_wait_timeout(1 << 26)
    with pytest.raises(L.FlbError) as e:
        sim.sync()
    assert e.value.code == L.FLB_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(L.FlbError) as e:                   # sticky for the life of the context
        sim.sync()
    assert e.value.code == L.FLB_ETIMEOUT
    sim.close()
    fresh = Sim(p, precision="fp32")
    fresh.run(3)
    fresh.sync()
    assert np.all(np.isfinite(fresh.populations()))
    fresh.close()

