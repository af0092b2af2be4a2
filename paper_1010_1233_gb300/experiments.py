"""The measured workloads beyond the headline bench: D1Q3 L = 64, D2Q9 256^2 spectra,
the 64-replica Galilean-invariance sweep and the learned-correction evaluation.

Each function runs one workload through the library and returns a dict of
results: throughput (MLUPS, wall time) and the correlator errors against the
ideal-gas values of Eq. 7 (delta_ab for the normalised spectra), the quantity
the paper's Figs. 1-4 show.  Wave vectors where the lattice has a neutral mode
(k = 0, and the momentum components at (pi, 0) / (0, pi), resp. pi in D1Q3)
are excluded.

    python -m paper_1010_1233_gb300.experiments d1q3 | d2q9_256 | sweep | learned [--quick]
"""
import json
import sys
import time

import numpy as np
import torch

from . import learned, workloads as W
from .sim import Sim


def _timed(sim, n, every):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.run(n, every)
    sim.sync()
    return time.perf_counter() - t0


def _mask(lattice, nx, ny):
    m = np.ones((ny, nx), bool)
    m[0, 0] = False
    if lattice == "D1Q3":
        m[0, nx // 2] = False
    else:
        m[0, nx // 2] = False
        m[ny // 2, 0] = False
    return m


def spectra_errors(sim, r, fields):
    """max |S_ab - delta_ab| over included k and all sampled pairs, and the k-average of it."""
    p = sim.params[r]
    ny = p["ny"] if p["lattice"] == "D2Q9" else 1
    km = _mask(p["lattice"], p["nx"], ny)
    worst, mean = 0.0, []
    for i, a in enumerate(fields):
        for b in fields[i:]:
            C = sim.correlator(r, a, b)[km]
            same = (a == b) or ({a, b} == {1, 9}) or ({a, b} == {2, 10})
            d = np.abs(C - (1.0 if same else 0.0))
            worst = max(worst, float(d.max()))
            mean.append(float(d.mean()))
    return worst, float(np.mean(mean))


def batched_errors(sim, steps, every, fields, batches=10, replicas=None):
    """Run `steps` in `batches` equal batches (statistics reset in between) and return
    (seconds, {r: (max |S - delta|, k-mean |S - delta|, max z)}) with the batch-means
    standard error sigma_k per point: z = |mean - delta| / sigma_k over the included k
    and all sampled pairs.  At u0 = 0, where Eq. 7 makes delta the exact answer, the z
    values measure the method against its statistical noise."""
    reps = range(len(sim.params)) if replicas is None else replicas
    per = max(1, steps // batches)
    samples = {r: {} for r in reps}
    t = 0.0
    for _ in range(batches):
        sim.reset_stats()
        t += _timed(sim, per, every)
        for r in reps:
            p = sim.params[r]
            ny = p["ny"] if p["lattice"] == "D2Q9" else 1
            km = _mask(p["lattice"], p["nx"], ny)
            for i, a in enumerate(fields):
                for b in fields[i:]:
                    samples[r].setdefault((a, b), []).append(sim.correlator(r, a, b)[km])
    out = {}
    for r in reps:
        worst, mean, zmax = 0.0, [], 0.0
        for (a, b), v in samples[r].items():
            v = np.array(v)
            m = v.mean(0)
            se = v.std(0, ddof=1) / np.sqrt(len(v))
            same = (a == b) or ({a, b} == {1, 9}) or ({a, b} == {2, 10})
            d = np.abs(m - (1.0 if same else 0.0))
            worst = max(worst, float(d.max()))
            mean.append(float(d.mean()))
            zmax = max(zmax, float((d / np.maximum(se, 1e-12)).max()))
        out[r] = (worst, float(np.mean(mean)), zmax)
    return t, out


def d1q3(steps=100_000, warmup=10_000, precision="fp64"):
    wl = W.d1q3_L64()
    p = wl["replicas"][0]
    sim = Sim(p, precision=precision)
    t_w = _timed(sim, warmup, 0)
    t, errs = batched_errors(sim, steps, 1, list(p["fields"]))
    mx, mean, z = errs[0]
    return dict(workload="d1q3_L64", precision=precision, steps=steps, warmup=warmup, wall_s=t + t_w,
                mlups=p["nx"] * steps / t / 1e6, max_err=mx, mean_err=mean, max_z=z, batches=10)


def d2q9_256(steps=200_000, warmup=10_000, precision="fp32", every=10):
    wl = W.d2q9_256()
    p = wl["replicas"][0]
    sim = Sim(p, precision=precision)
    sim.autotune(3)
    _timed(sim, warmup, 0)
    t, errs = batched_errors(sim, steps, every, list(p["fields"]))
    mx, mean, z = errs[0]
    V = p["nx"] * p["ny"]
    return dict(workload="d2q9_256", precision=precision, steps=steps, sample_every=every, wall_s=t,
                mlups=V * steps / t / 1e6, samples=steps // every, max_err=mx, mean_err=mean, max_z=z,
                batches=10)


def sweep(steps=100_000, warmup=10_000, every=10):
    wl = W.sweep64()
    reps = wl["replicas"]
    sim = Sim(reps, precision="fp32")
    vec, grid, staged, _ = sim.autotune(3)
    _timed(sim, warmup, 0)
    fields = list(reps[0]["fields"])
    t, errs = batched_errors(sim, steps, every, fields)
    V = sum(p["nx"] * p["ny"] for p in reps)
    rows = []
    for r, p in enumerate(reps):
        c = sim.conserved(r)
        finite = bool(np.all(np.isfinite(c)))
        mx, mean, z = errs[r] if finite else (float("nan"),) * 3
        rows.append(dict(r=r, n=p["nx"], u0=p["u0"][0], tau_s=p["tau"][3], max_err=mx, mean_err=mean,
                         max_z=z, finite=finite))
    return dict(workload="sweep64", steps=steps, sample_every=every, sites=V, wall_s=t, mlups=V * steps / t / 1e6,
                launch=dict(vec=vec, grid=grid, staged=staged), replicas=rows)


def learned_eval(quick=False):
    kw = dict(n=32, n_train=4, steps=20_000, warmup=2_000, sample_every=5, iters=600) if quick else {}
    res, _ = learned.experiment(**kw)
    return res


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "d1q3"
    quick = "--quick" in sys.argv
    if which == "d1q3":
        out = d1q3(**(dict(steps=10_000, warmup=1_000) if quick else {}))
    elif which == "d2q9_256":
        prec = "fp64" if "--fp64" in sys.argv else "fp32"
        out = d2q9_256(precision=prec, **(dict(steps=20_000, warmup=1_000) if quick else {}))
    elif which == "sweep":
        out = sweep(**(dict(steps=2_000, warmup=200) if quick else {}))
    elif which == "learned":
        out = learned_eval(quick)
    else:
        raise SystemExit(f"unknown workload {which}")
    print(json.dumps(out))
