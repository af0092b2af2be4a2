"""CUDA path against the FP64 oracle, element by element, through the C ABI (GPU)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import lb, mlp as omlp, philox as ophilox, spectra
from paper_1010_1233_gb300 import Sim, philox, workloads as W
from paper_1010_1233_gb300 import _lib as L

pytestmark = pytest.mark.gpu

LADD = (1 << 3) | (1 << 4) | (1 << 5)
FP64_TOL = 1e-12        # per step, relative to max |f - w rho0|
FP32_TOL = 2e-5         # after the run, relative to max |f - w rho0|


def _oracle(p, **kw):
    d = dict(p)
    d.update(kw)
    return lb.Run(lb.Params(**d))


def _rel(a, b, ref):
    """max |a - b| relative to max |ref| (ref = the oracle's deviation from equilibrium)."""
    return np.abs(a - b).max() / max(np.abs(ref).max(), 1e-12)


# ---------------------------------------------------------------------------- generator
def test_philox_words_bit_exact_and_normals():
    rng = np.random.default_rng(1)
    sites = np.concatenate([np.arange(1000), rng.integers(0, 2**32, 3000)]).astype(np.uint32)
    for step, call, tag, stream, seed in [(0, 0, 0, 0, 0), (123456, 1, 0, 5, 7), (2**32 - 1, 2, 1, 63, 2**64 - 3)]:
        words, nrm = philox(sites, step, call, tag, stream, seed)
        want = ophilox.philox4x32_10(sites.astype(np.uint64), step, call | (tag << 8), stream, seed)
        for k in range(4):
            assert np.array_equal(words[:, k], want[k])
        a0, a1 = ophilox.box_muller(ophilox.uniform_fp64(want[0]), ophilox.uniform_fp64(want[1]))
        a2, a3 = ophilox.box_muller(ophilox.uniform_fp64(want[2]), ophilox.uniform_fp64(want[3]))
        ref = np.stack([a0, a1, a2, a3], 1)
        assert np.abs(nrm - ref).max() < 1e-13
        # FP32 recipe: 23-bit uniforms, single-precision log/sincos
        _, n32 = philox(sites, step, call, tag, stream, seed, fp32=True)
        assert np.abs(n32 - ref).max() < 1e-4
        assert np.median(np.abs(n32 - ref)) < 2e-6


# ---------------------------------------------------------------------------- FP64 step
CASES = [
    ("D2Q9", 64, 64, dict(tau=W.taus_d2q9(0.8, 0.8, 1.0), u0=(0.0, 0.0), init_mode=1)),
    ("D2Q9", 128, 32, dict(tau=W.taus_d2q9(0.6, 0.9, 1.3), u0=(0.1, 0.05), init_mode=1)),
    ("D2Q9", 24, 10, dict(tau=W.taus_d2q9(0.7, 0.7, 1.0), u0=(-0.05, 0.1), noise_mask=LADD)),
    ("D1Q3", 64, 1, dict(tau=W.taus_d1q3(0.8), init_mode=1)),
    ("D1Q3", 22, 1, dict(tau=W.taus_d1q3(0.55), u0=(0.2, 0.0))),
]


@pytest.mark.parametrize("lat,nx,ny,kw", CASES, ids=[f"{c[0]}-{c[1]}x{c[2]}" for c in CASES])
def test_fp64_step_matches_oracle_every_step(lat, nx, ny, kw):
    p = W.replica(lat, nx, ny, kT=1e-3, seed=11, stream=3, **kw)
    sim = Sim(p, precision="fp64")
    ref = _oracle(p)
    feq = lb.uniform_state(ref.p)
    assert np.abs(sim.populations() - ref.f).max() < 1e-15 * np.abs(ref.f).max()
    worst = 0.0
    for _ in range(100):
        sim.run(1)
        ref.run(1)
        worst = max(worst, _rel(sim.populations(), ref.f, ref.f - feq))
    assert worst < FP64_TOL, worst
    c = sim.conserved()
    assert abs(c[0] - ref.conserved()[0]) < 1e-12 * nx * ny


def test_fp64_from_arbitrary_state():
    p = W.replica("D2Q9", 32, 16, W.taus_d2q9(0.9, 0.7, 1.5), kT=1e-2, u0=(0.03, -0.02), seed=3)
    ref = _oracle(p)
    f = ref.f * (1 + W.random_perturbation(ref.f.shape, 8, 0.02))
    ref = _oracle(p)
    ref.f = f.copy()
    sim = Sim(p, precision="fp64")
    sim.set_populations(f)
    sim.run(30)
    ref.run(30)
    assert _rel(sim.populations(), ref.f, ref.f - lb.uniform_state(ref.p)) < FP64_TOL


# ---------------------------------------------------------------------------- FP32 deviation storage
@pytest.mark.parametrize("nx,ny", [(64, 64), (36, 20), (30, 8)])
def test_fp32_dev_close_to_oracle(nx, ny):
    p = W.replica("D2Q9", nx, ny, W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, u0=(0.1, 0.05), seed=4,
                  init_mode=1)
    sim = Sim(p, precision="fp32")
    ref = _oracle(p)
    feq = lb.uniform_state(ref.p)
    errs = []
    for _ in range(10):
        sim.run(10)
        ref.run(10)
        errs.append(_rel(sim.populations(), ref.f, ref.f - feq))
    print("FP32-dev relative population error every 10 steps:", ["%.1e" % e for e in errs])
    assert max(errs) < FP32_TOL


# ---------------------------------------------------------------------------- correlators
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_correlators_match_oracle(precision, tol):
    fields = (0, 1, 2, 3, 5, 8, W.FIELD_UX, W.FIELD_UY)
    p = W.replica("D2Q9", 16, 32, W.taus_d2q9(0.8, 0.9, 1.1), kT=1e-3, u0=(0.08, -0.04), seed=21,
                  init_mode=1, fields=fields)
    sim = Sim(p, precision=precision)
    ref = _oracle(p)
    sim.run(40, sample_every=3)
    ref.run(40, sample_every=3)
    for a, b in spectra.pairs(fields):
        g, n = sim.correlator(0, a, b, with_count=True)
        o = ref.acc.correlator(a, b)
        assert n == ref.acc.n
        err = np.abs(g - o).max() / max(1.0, np.abs(o).max())
        assert err < tol, (a, b, err)


def test_d1q3_correlators_match_oracle():
    p = W.replica("D1Q3", 64, 1, W.taus_d1q3(0.8), kT=1e-4, seed=1, init_mode=1, fields=(0, 1, 2, 9))
    sim = Sim(p, precision="fp64")
    ref = _oracle(p)
    sim.run(50, 1)
    ref.run(50, 1)
    for a, b in spectra.pairs(p["fields"]):
        assert np.abs(sim.correlator(0, a, b) - ref.acc.correlator(a, b)).max() < 1e-9


@pytest.mark.parametrize("nx,ny", [(64, 256), (16, 4096)])
def test_folded_samples_equal_single_sample_passes(nx, ny):
    # FP32 with register-resident columns (one pass of 256; four-step 64 x 64) folds two
    # samples into one pass over the FP64 sums (spectrum slots 0 and 1).  Each sum still
    # gets the first sample's product added and then the second's, so one run of all the
    # steps (pairs inside the captured chunks, a lone last sample at the end) must give
    # the same sums, bit for bit, as one-step runs (a run leaves no sample waiting, so
    # every sample there gets a pass of its own).
    fields = (0, 3, W.FIELD_UX, W.FIELD_UY)
    p = W.replica("D2Q9", nx, ny, W.taus_d2q9(0.7, 0.8, 1.1), kT=1e-3, u0=(0.05, 0.02), seed=41, init_mode=1,
                  fields=fields)
    a = Sim(p, precision="fp32")
    a.run(133, 4)                      # graph chunks of 32 steps (8 samples), then direct steps
    b = Sim(p, precision="fp32")
    b.set_graphs(False)
    for _ in range(133):
        b.run(1, 4)
    assert np.array_equal(a.populations(), b.populations())
    for x, y in spectra.pairs(fields):
        ga, na = a.correlator(0, x, y, with_count=True)
        gb, nb = b.correlator(0, x, y, with_count=True)
        assert na == nb == 34
        assert np.array_equal(ga, gb), (x, y)
    a.close()
    b.close()


def test_kernel_launch_count():
    # flb_kernel_launches (the count bench.py reports as gpu_launches) against the schedule
    # flb_run follows: one step kernel per step; per sample the row transform (16-point rows:
    # the shared-memory kernel) and, every second sample and at the end of a run, one
    # accumulation pass (16-point columns: the register-resident kernel, two samples folded)
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8), kT=1e-4, seed=3, init_mode=1,
                  fields=(0, W.FIELD_UX, W.FIELD_UY))
    sim = Sim(p, precision="fp32")
    sim.set_graphs(False)
    n0 = sim.kernel_launches()
    sim.run(3, 1)                          # 3 steps, 3 row passes, accumulations after samples 2 and 3
    assert sim.kernel_launches() - n0 == 3 + 3 + 2
    sim.set_graphs(True)
    n0 = sim.kernel_launches()
    sim.run(64, 1)                         # from step 3: 29 direct steps, then a 32-step chunk
    direct = 29 + 29 + 15                  # steps, row passes, the (29 + 1) / 2 accumulations
    chunk = 32 + 32 + 16 + 1               # steps, row passes, accumulations, step-counter advance
    assert sim.kernel_launches() - n0 == direct + 1 + chunk + 3 + 3 + 2
    sim.close()


# ---------------------------------------------------------------------------- batching, checkpoint
def test_batched_replicas_equal_single():
    # a batched launch runs each replica exactly as a launch of that replica alone: the
    # one-replica launch is a separate kernel instantiation (description in the constant
    # bank), but the site update is written with explicitly rounded operations (nothing
    # left to multiply-add contraction), so the two agree bit for bit.  Two runs of the
    # same batch are bitwise identical too (no atomics in the step or the correlator sums).
    reps = [W.replica("D2Q9", 32, 32, W.taus_d2q9(0.7 + 0.1 * i), kT=1e-4, u0=(0.02 * i, 0), seed=i,
                      stream=i, init_mode=1, fields=(0, 9, 10)) for i in range(3)]
    reps.append(W.replica("D2Q9", 64, 16, W.taus_d2q9(0.9), kT=1e-4, seed=9, stream=9, fields=(0, 9, 10)))
    for prec in ("fp64", "fp32"):
        batch = Sim(reps, precision=prec)
        batch.run(25, 5)
        again = Sim(reps, precision=prec)
        again.run(25, 5)
        for i, p in enumerate(reps):
            assert np.array_equal(batch.populations(i), again.populations(i))
            assert np.array_equal(batch.correlator(i, 0, 9), again.correlator(i, 0, 9))
            one = Sim(p, precision=prec)
            one.run(25, 5)
            assert np.array_equal(batch.populations(i), one.populations()), (prec, i)
            for a, b in ((0, 0), (0, 9), (9, 10)):
                assert np.array_equal(batch.correlator(i, a, b), one.correlator(0, a, b)), (prec, i, a, b)


def test_checkpoint_resume_bitwise():
    p = W.replica("D2Q9", 32, 32, W.taus_d2q9(0.8), kT=1e-4, seed=2, init_mode=1, fields=(0, 9))
    a = Sim(p, precision="fp32")
    a.run(20, 4)
    blob = a.save()
    a.run(20, 4)
    b = Sim(p, precision="fp32")
    b.load(blob)
    assert b.step == 20
    b.run(20, 4)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.correlator(0, 0, 9), b.correlator(0, 0, 9))


def test_conservation_fp64_long_run():
    p = W.replica("D2Q9", 64, 64, W.taus_d2q9(0.55, 0.6, 1.9), kT=1e-3, u0=(0.1, 0.1), seed=5, init_mode=1)
    sim = Sim(p, precision="fp64")
    c0 = sim.conserved()
    sim.run(2000)
    assert np.abs(sim.conserved() - c0).max() < 1e-13 * 64 * 64


# ---------------------------------------------------------------------------- noise-scale network
NET_CASES = [("warp", 2, 32, 16), ("warp", 1, 32, 16), ("warp", 4, 32, 16), ("warp", 2, 70, 9), ("warp", 1, 34, 5),
             ("tcgen05", 2, 32, 16), ("tcgen05", 1, 70, 9)]


@pytest.mark.parametrize("engine,vec,nx,ny", NET_CASES, ids=[f"{c[0]}-v{c[1]}-{c[2]}x{c[3]}" for c in NET_CASES])
def test_mlp_scaled_noise_matches_oracle(engine, vec, nx, ny):
    # both network engines at every vector width; ragged rows (70 = 2 warps + 6 sites at
    # vec 1, 34 = one warp + 2 sites at vec 1) leave warps with inactive lanes, which still take part in
    # the warp-level MMAs
    wts = W.mlp_weights(3, out_scale=0.5)
    p = W.replica("D2Q9", nx, ny, W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, u0=(0.15, -0.05), seed=6,
                  init_mode=1)
    sim = Sim(p, precision="fp32")
    sim.set_mlp(wts)
    sim.set_network_engine(engine)
    assert sim.network_engine() == engine
    if nx % vec == 0:
        sim.set_step_config(vec, 0, 0)
    w64 = {k: (omlp.to_bf16(v) if k.startswith("W") else v.astype(np.float64)) for k, v in wts.items()}
    ref = _oracle(p)
    ref.p.mlp = w64
    ref.p.mlp_bf16 = True
    sim.run(10)
    ref.run(10)
    feq = lb.uniform_state(ref.p)
    err = _rel(sim.populations(), ref.f, ref.f - feq)
    # Both sides round the network's operands to bfloat16, but from FP32 (kernel) and FP64
    # (oracle) pre-activations: a value within ~1e-7 of a rounding tie can round to the
    # neighbouring bfloat16 (one ulp, 2^-8..2^-7 relative).  One such flip moves s_c by
    # |W3| ulp(h) ~ 0.09 * 0.008 ~ 7e-4 at one site, i.e. ~1e-4 of the maximal deviation.
    assert err < 1e-3, err
    # the network really changes the dynamics
    plain = _oracle(p)
    plain.run(10)
    assert _rel(plain.f, ref.f, ref.f - feq) > 20 * err


STAGED = [(260, 6, 1, False), (264, 5, 2, True), (512, 4, 1, True), (64, 8, 4, False), (1032, 3, 4, True),
          (16, 8, 2, True), (1024, 2, 4, False)]


@pytest.mark.parametrize("nx,ny,vec,with_mlp", STAGED, ids=[f"{c[0]}x{c[1]}-v{c[2]}-{'mlp' if c[3] else 'plain'}"
                                                           for c in STAGED])
def test_staged_kernel_matches_oracle(nx, ny, vec, with_mlp):
    # row tiles of 256 vec sites through shared memory: full tiles, ragged last tiles
    # (260 = 256 + 4, 1032 = 1024 + 8), rows shorter than one warpgroup's half (16, 64),
    # and the periodic halos at both row ends; on power-of-two lattices also the sampled
    # fields and correlators (every 3 steps)
    pow2 = (nx & (nx - 1)) == 0 and (ny & (ny - 1)) == 0
    fields = (0, 9, 10) if pow2 else ()
    p = W.replica("D2Q9", nx, ny, W.taus_d2q9(0.8, 0.7, 1.1), kT=1e-4, u0=(0.12, -0.04), seed=8,
                  init_mode=1, fields=fields)
    sim = Sim(p, precision="fp32")
    ref = _oracle(p)
    tol = FP32_TOL
    if with_mlp:
        wts = W.mlp_weights(3, out_scale=0.5)
        sim.set_mlp(wts)
        ref.p.mlp = {k: (omlp.to_bf16(v) if k.startswith("W") else v.astype(np.float64)) for k, v in wts.items()}
        ref.p.mlp_bf16 = True
        tol = 1e-3          # bfloat16 rounding ties, see test_mlp_scaled_noise_matches_oracle
    sim.set_step_config(vec, 0, 1)
    assert sim.step_config()[2] == 1
    sim.run(12, 3 if pow2 else 0)
    ref.run(12, 3 if pow2 else 0)
    feq = lb.uniform_state(ref.p)
    assert _rel(sim.populations(), ref.f, ref.f - feq) < tol
    for a, b in spectra.pairs(fields):
        g, o = sim.correlator(0, a, b), ref.acc.correlator(a, b)
        assert np.abs(g - o).max() < 5 * tol * max(1.0, np.abs(o).max()), (a, b)


def test_mlp_zero_output_is_plain_method_bitwise():
    wts = W.mlp_weights(4)
    wts["W3"][:] = 0
    wts["b3"][:] = 0
    p = W.replica("D2Q9", 32, 32, W.taus_d2q9(0.8), kT=1e-4, u0=(0.1, 0), seed=7, init_mode=1)
    a = Sim(p, precision="fp32")
    a.set_mlp(wts)
    b = Sim(p, precision="fp32")
    a.run(15)
    b.run(15)
    assert np.array_equal(a.populations(), b.populations())


def test_errors_surface_without_fault():
    p = W.replica("D2Q9", 16, 16, fields=(0,))
    sim = Sim(p, precision="fp32")
    with pytest.raises(L.FlbError):
        sim.correlator(0, 0, 0)         # no samples yet
    with pytest.raises(L.FlbError):
        sim.correlator(0, 0, 9)         # field 9 not sampled
    with pytest.raises(L.FlbError):
        sim.populations(3)              # replica out of range
    buf = np.zeros(9 * 16 * 16)
    rc = L.lib().flb_get_populations(sim._ctx, 3, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == L.FLB_EINVAL and not buf.any()
    assert L.lib().flb_run(sim._ctx, 1, 0) == 0 and sim.step == 1


@pytest.mark.parametrize("precision,nx,ny,tol", [("fp64", 8, 2048, 1e-10), ("fp32", 8, 4096, 2e-4)])
def test_four_step_column_fft_matches_oracle(precision, nx, ny, tol):
    # columns too long for shared memory take the N1 x N2 split
    fields = (0, W.FIELD_UX, W.FIELD_UY)
    p = W.replica("D2Q9", nx, ny, W.taus_d2q9(0.7, 0.8, 1.2), kT=1e-3, u0=(0.05, 0.1), seed=31,
                  init_mode=1, fields=fields)
    sim = Sim(p, precision=precision)
    ref = _oracle(p)
    sim.run(6, sample_every=2)
    ref.run(6, sample_every=2)
    for a, b in spectra.pairs(fields):
        o = ref.acc.correlator(a, b)
        err = np.abs(sim.correlator(0, a, b) - o).max() / max(1.0, np.abs(o).max())
        assert err < tol, (a, b, err)


@pytest.mark.parametrize("with_mlp", [False, True])
def test_step_configs_and_autotune(with_mlp):
    # every launch configuration computes the same step; the template variants may contract
    # multiply-adds differently, so agreement is to FP32 rounding, not bitwise
    # (with the network: per engine; across engines the FP32 accumulation order of the
    # network differs, so a bfloat16 rounding tie can flip: the network tolerance 1e-3)
    p = W.replica("D2Q9", 64, 32, W.taus_d2q9(0.8), kT=1e-4, u0=(0.1, 0.02), seed=12, init_mode=1,
                  fields=(0, 9, 10))
    wts = W.mlp_weights(5, out_scale=0.3)
    ref, refs = None, {}
    feq = lb.uniform_state(lb.Params(**p))
    engines = ("warp", "tcgen05") if with_mlp else ("warp",)
    for engine in engines:
        for vec, grid, staged in [(4, 0, 0), (1, 0, 0), (2, 3, 0), (4, 1, 0), (1, 100000, 0),
                                  (1, 0, 1), (2, 0, 1), (4, 0, 1), (2, 1, 1)]:
            sim = Sim(p, precision="fp32")
            if with_mlp:
                sim.set_mlp(wts)
                sim.set_network_engine(engine)
            sim.set_step_config(vec, grid, staged)
            assert sim.step_config()[0] == vec and sim.step_config()[2] == staged
            sim.run(12, 4)
            out = (sim.populations(), sim.correlator(0, 0, 9))
            key = "tcgen05" if staged else engine          # the staged kernel's network is tcgen05
            if ref is None:
                ref = out
            if key not in refs:
                refs[key] = out
            r0 = refs[key]
            assert _rel(out[0], r0[0], r0[0] - feq) < 1e-5, (engine, vec, grid, staged)
            assert np.abs(out[1] - r0[1]).max() < 1e-4 * np.abs(r0[1]).max(), (engine, vec, grid, staged)
            assert _rel(out[0], ref[0], ref[0] - feq) < (1e-3 if with_mlp else 1e-5), (engine, vec, grid, staged)
    # the autotuner's timing launches leave the state and the step counter unchanged
    sim = Sim(p, precision="fp32")
    if with_mlp:
        sim.set_mlp(wts)
    sim.run(6, 4)
    before, step = sim.populations(), sim.step
    vec, grid, staged, ms = sim.autotune(trials=3)
    assert vec in (1, 2, 4) and grid > 0 and staged in (0, 1) and ms > 0
    assert np.array_equal(sim.populations(), before) and sim.step == step
    sim.run(6, 4)
    assert _rel(sim.populations(), ref[0], ref[0] - feq) < (1e-3 if with_mlp else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("every", [0, 1, 3])
def test_d1q3_fused_launch_matches_per_step_launches(precision, every):
    """D1Q3 runs of steps go through one fused launch (state, fields and row transforms in
    shared memory); with graphs off every step and every sample is launched separately.
    Uneven replicas, one without fields; starts at odd and even steps.  The two paths do
    the same arithmetic in the same order (they may differ in multiply-add contraction)."""
    reps = [W.replica("D1Q3", 64, 1, W.taus_d1q3(0.8), kT=1e-4, seed=1, init_mode=1, fields=(0, 1, 2, 9)),
            W.replica("D1Q3", 256, 1, W.taus_d1q3(0.6), kT=1e-4, u0=(0.1, 0.0), seed=2, stream=1, init_mode=1,
                      fields=(1,)),
            W.replica("D1Q3", 30, 1, W.taus_d1q3(0.7), kT=1e-4, seed=3, stream=2, init_mode=1),
            W.replica("D1Q3", 4, 1, W.taus_d1q3(0.9), kT=1e-4, seed=4, stream=3, init_mode=1, fields=(0, 2))]
    a, b = Sim(reps, precision=precision), Sim(reps, precision=precision)
    b.set_graphs(False)
    for n in (5, 100, 7):
        a.run(n, every)
        b.run(n, every)
    assert a.step == b.step == 112
    tol = 1e-13 if precision == "fp64" else 2e-6
    for r, p in enumerate(reps):
        fa, fb = a.populations(r), b.populations(r)
        feq = lb.uniform_state(lb.Params(**p))
        assert _rel(fa, fb, fb - feq) < tol, r
        fl = list(p["fields"])
        if every and fl:                           # the fields of the last sample (step 111 or 110)
            assert np.abs(a.fields(r) - b.fields(r)).max() < tol * max(1e-3, np.abs(b.fields(r)).max()), r
        for i, x in enumerate(fl if every else []):
            for y in fl[i:]:
                ca, na = a.correlator(r, x, y, with_count=True)
                cb, nb = b.correlator(r, x, y, with_count=True)
                assert na == nb == len(range(0, 112, every))
                assert np.abs(ca - cb).max() < tol * max(1.0, np.abs(cb).max()), (r, x, y)


@pytest.mark.parametrize("every", [0, 4, 5])
def test_graph_replay_bitwise_equal_direct(every):
    reps = [W.replica("D2Q9", 32, 16, W.taus_d2q9(0.8), kT=1e-4, u0=(0.05, 0), seed=3, init_mode=1,
                      fields=(0, 9, 10)),
            W.replica("D2Q9", 16, 16, W.taus_d2q9(0.7), kT=1e-4, seed=4, stream=1, fields=(0, 9, 10))]
    a, b = Sim(reps, precision="fp32"), Sim(reps, precision="fp32")
    b.set_graphs(False)
    for n in (3, 70, 9):                      # unaligned start, replayed chunks, tail
        a.run(n, every)
        b.run(n, every)
    assert a.step == b.step == 82
    for r in range(2):
        assert np.array_equal(a.populations(r), b.populations(r))
        if every:
            ca, na = a.correlator(r, 0, 9, with_count=True)
            cb, nb = b.correlator(r, 0, 9, with_count=True)
            assert na == nb and np.array_equal(ca, cb)
