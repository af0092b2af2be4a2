"""The bounds-checked debug build (GPU).

The library is built a second time with every computed global and shared-memory
index checked (-DFLB_CHECK_BOUNDS: a violation is counted and the access skipped,
never trapped), and a child process runs small and ragged cases through it against
the FP64 oracle: D2Q9 FP64 and FP32 at 8^2 .. 16^2 with sampling, rows of 10 and 14
sites (vec 1 and 2), a single-row lattice, both network engines at vec 1/2/4,
uneven batched replicas, the four-step column transform, the Stockham row pass with
the column-tiled spectrum (a 4096 x 64 lattice, and the standalone sampler on a 4096^2
field at sampled wave vectors), D1Q3 (fused and per step) and D3Q15 / D3Q19 boxes
with time correlators.  Every case must match the oracle and
the run must end with zero violations.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, %r)
from paper_1010_1233_gb300 import _lib as L, Sim, workloads as W
assert L.LIB_PATH.endswith("libflb_checked.so")
from oracle import lb, lb3d, mlp as omlp, spectra
import ctypes

def viol():
    n, site = ctypes.c_uint64(), ctypes.c_uint32()
    L.check(L.lib().flb_debug_bounds(ctypes.byref(n), ctypes.byref(site), 1))
    return int(n.value), int(site.value)

out = {}
def rel(a, b, ref):
    return float(np.abs(a - b).max() / max(np.abs(ref).max(), 1e-12))

def d2q9(name, p, prec, steps, every, tol, vec=None, engine=None, mlp=False):
    sim = Sim(p, precision=prec)
    ref = lb.Run(lb.Params(**p))
    if mlp:
        wts = W.mlp_weights(3, out_scale=0.5)
        sim.set_mlp(wts)
        ref.p.mlp = {k: (omlp.to_bf16(v) if k.startswith("W") else v.astype(np.float64)) for k, v in wts.items()}
        ref.p.mlp_bf16 = True
    if engine:
        sim.set_network_engine(engine)
    if vec:
        sim.set_step_config(vec, 0, 0)
    sim.run(steps, every)
    ref.run(steps, every)
    err = rel(sim.populations(), ref.f, ref.f - lb.uniform_state(ref.p))
    cerr = 0.0
    if every and p["fields"]:
        for a, b in spectra.pairs(p["fields"]):
            o = ref.acc.correlator(a, b)
            cerr = max(cerr, float(np.abs(sim.correlator(0, a, b) - o).max() / max(1.0, np.abs(o).max())))
    sim.close()
    out[name] = dict(err=err, cerr=cerr, ok=bool(err < tol and cerr < 10 * tol), viol=viol())

F3 = (0, W.FIELD_UX, W.FIELD_UY)
d2q9("fp64_8x8", W.replica("D2Q9", 8, 8, W.taus_d2q9(0.8, 0.9, 1.2), kT=1e-3, u0=(0.05, 0.02), seed=5,
     init_mode=1, fields=F3), "fp64", 6, 1, 1e-12)
d2q9("fp32_16x16", W.replica("D2Q9", 16, 16, W.taus_d2q9(0.7), kT=1e-4, u0=(0.1, 0.0), seed=6, init_mode=1,
     fields=tuple(range(9))), "fp32", 8, 2, 2e-5)
d2q9("fp32_10x6_v1", W.replica("D2Q9", 10, 6, W.taus_d2q9(0.8), kT=1e-4, seed=7, init_mode=1), "fp32", 8, 0, 2e-5, vec=1)
d2q9("fp32_14x5_v2", W.replica("D2Q9", 14, 5, W.taus_d2q9(0.8), kT=1e-4, seed=8, init_mode=1), "fp32", 8, 0, 2e-5, vec=2)
d2q9("fp32_16x1_row", W.replica("D2Q9", 16, 1, W.taus_d2q9(0.8), kT=1e-4, seed=9, init_mode=1, fields=F3),
     "fp32", 8, 2, 2e-5)
for eng in ("warp", "tcgen05"):
    for v in (1, 2, 4):
        d2q9(f"net_{eng}_v{v}", W.replica("D2Q9", 16, 8, W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, u0=(0.15, -0.05),
             seed=6, init_mode=1, fields=F3), "fp32", 6, 3, 1e-3, vec=v, engine=eng, mlp=True)
d2q9("fourstep_8x4096", W.replica("D2Q9", 8, 4096, W.taus_d2q9(0.7, 0.8, 1.2), kT=1e-3, u0=(0.05, 0.1), seed=31,
     init_mode=1, fields=F3), "fp32", 4, 2, 2e-4)

# the Stockham row pass (rows of 4096) with column-tiled spectra, one-pass columns of 64
d2q9("rows16_4096x64", W.replica("D2Q9", 4096, 64, W.taus_d2q9(0.7, 0.8, 1.2), kT=1e-3, u0=(0.05, 0.1), seed=33,
     init_mode=1, fields=F3), "fp32", 3, 1, 2e-4)

# the standalone sampler on a 4096^2 field: Stockham rows, tiled spectrum, both
# register-resident four-step passes (64 x 64), checked at sampled wave vectors
import torch
from paper_1010_1233_gb300.sim import spectra_accumulate, unpack_pair_sums
x = W.random_perturbation((1, 4096, 4096), 44) + 0.3
sums, mean0 = spectra_accumulate(torch.tensor(x, dtype=torch.float32, device="cuda"))
g = unpack_pair_sums(sums, 1, 4096, 4096)[(0, 0)]
xr = np.asarray(torch.tensor(x, dtype=torch.float32).double())[0]
err = 0.0
for ky, kx in [(0, 0), (1, 1), (4095, 2048), (2048, 1024), (3, 5), (1234, 777)]:
    want = abs(spectra.dft_at(xr, kx, ky)) ** 2
    err = max(err, abs(g[ky, kx] - want) / max(want, 1.0))
out["spectra_4096sq"] = dict(err=err, ok=bool(err < 1e-4), viol=viol())

# uneven batched replicas against single-replica oracle runs
reps = [W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8), kT=1e-4, seed=1, stream=1, init_mode=1, fields=F3),
        W.replica("D2Q9", 8, 8, W.taus_d2q9(0.9), kT=1e-4, u0=(0.1, 0), seed=2, stream=2, init_mode=1, fields=F3)]
sim = Sim(reps, precision="fp32")
sim.run(6, 3)
err = 0.0
for i, p in enumerate(reps):
    ref = lb.Run(lb.Params(**p)); ref.run(6, 3)
    err = max(err, rel(sim.populations(i), ref.f, ref.f - lb.uniform_state(ref.p)))
sim.close()
out["batched"] = dict(err=err, ok=bool(err < 2e-5), viol=viol())

# D1Q3: fused runs (graphs on) and per-step launches (graphs off)
for graphs in (True, False):
    p = W.replica("D1Q3", 16, 1, W.taus_d1q3(0.8), kT=1e-3, seed=1, init_mode=1, fields=(0, 1, 2))
    sim = Sim(p, precision="fp64")
    sim.set_graphs(graphs)
    ref = lb.Run(lb.Params(**p))
    sim.run(40, 1); ref.run(40, 1)
    err = rel(sim.populations(), ref.f, ref.f - lb.uniform_state(ref.p))
    sim.close()
    out[f"d1q3_graphs{int(graphs)}"] = dict(err=err, ok=bool(err < 1e-12), viol=viol())

# 3D boxes with time correlators at a few wave vectors
for lat in ("D3Q15", "D3Q19"):
    tau = W.taus_d3q15(0.7, 0.9, 1.1) if lat == "D3Q15" else W.taus_d3q19(0.7, 0.9, 1.1)
    q = W.replica3(8, 6, 4, tau, kT=1e-3, u0=(0.05, -0.02, 0.03), seed=9, init_mode=1, lattice=lat, fields=(0, 4))
    sim = Sim(q, precision="fp32")
    sim.set_time_correlator([(0, 0, 1), (1, 2, 3)], 2)
    ref = lb3d.Run3(lb3d.Params3(nx=8, ny=6, nz=4, tau=q["tau"], rho0=q["rho0"], kT=q["kT"], u0=q["u0"],
                                 seed=q["seed"], stream=q["stream"], init_mode=1, fields=[0, 4], lattice=lat))
    sim.run(5, 1); ref.run(5, 1)
    err = rel(sim.populations(), ref.f, ref.f - lb3d.uniform_state(ref.p))
    sim.close()
    out[lat] = dict(err=err, ok=bool(err < 2e-5), viol=viol())

print(json.dumps(out))
""" % ROOT


def test_checked_build_matches_oracle_without_violations():
    from paper_1010_1233_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, FLB_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, env=env, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    bad = {k: v for k, v in res.items() if not v["ok"] or v["viol"][0] != 0}
    assert not bad, bad
    assert len(res) >= 18
