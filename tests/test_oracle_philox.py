"""Pins of the oracle's Philox4x32-10 and Box-Muller (CPU only).

The bit-exact pin runs an installed, independent Philox4x32-10 (Triton's,
executed by its CPU interpreter) in a subprocess and compares every word.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

from oracle import philox as P

_TRITON_SCRIPT = r"""
import os, json, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(out_ptr, c0p, c1p, c2p, c3p, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    r0, r1, r2, r3 = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i),
                               tl.load(c2p + i), tl.load(c3p + i))
    tl.store(out_ptr + 4 * i + 0, r0); tl.store(out_ptr + 4 * i + 1, r1)
    tl.store(out_ptr + 4 * i + 2, r2); tl.store(out_ptr + 4 * i + 3, r3)

req = json.loads(sys.stdin.read())
res = []
for case in req:
    c = [torch.tensor(np.array(x, dtype=np.uint32).view(np.int32)) for x in case["c"]]
    N = len(case["c"][0])
    out = torch.zeros(4 * N, dtype=torch.int32)
    k[(1,)](out, *c, case["seed"], N=N)
    res.append(out.numpy().view(np.uint32).reshape(N, 4).T.tolist())
print(json.dumps(res))
"""


def _triton_available():
    try:
        import triton  # noqa: F401
        return True
    except Exception:
        return False


@pytest.mark.skipif(not _triton_available(), reason="triton not installed")
def test_philox_matches_independent_implementation():
    rng = np.random.default_rng(5)
    cases = []
    N = 64
    for seed in (0, 1, 7, 0x123456789ABCDEF, 2**63 + 12345):
        c = [rng.integers(0, 2**32, N, dtype=np.uint64) for _ in range(4)]
        c[0][:4] = [0, 1, 2, 2**32 - 1]
        c[1][:4] = [0, 0, 5, 2**32 - 1]
        cases.append(dict(seed=int(seed), c=[x.tolist() for x in c]))
    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                         capture_output=True, text=True, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for case, want in zip(cases, ref):
        got = P.philox4x32_10(*[np.array(x, dtype=np.uint64) for x in case["c"]], case["seed"])
        for w_got, w_want in zip(got, want):
            assert np.array_equal(w_got.astype(np.uint64), np.array(w_want, dtype=np.uint64))


def test_philox_words_uniform_and_decorrelated():
    site = np.arange(200_000, dtype=np.uint64)
    w = P.philox4x32_10(site, 3, 0, 0, seed=42)
    for x in w:
        # bytes uniform
        b = (x.astype(np.uint64) & np.uint64(0xFF)).astype(np.int64)
        chi2 = stats.chisquare(np.bincount(b, minlength=256)).pvalue
        assert chi2 > 1e-4
        assert abs(x.astype(np.float64).mean() / 2**32 - 0.5) < 0.005
    # neighbouring counters and different words are uncorrelated
    u = [P.uniform_fp64(x) for x in w]
    assert abs(np.corrcoef(u[0][:-1], u[0][1:])[0, 1]) < 0.01
    assert abs(np.corrcoef(u[0], u[1])[0, 1]) < 0.01
    # changing the step word changes every output
    w2 = P.philox4x32_10(site[:1000], 4, 0, 0, seed=42)
    assert np.mean(w2[0] == w[0][:1000]) < 0.01


def test_uniform_range_exact():
    u = P.uniform_fp64(np.array([0, 2**32 - 1], dtype=np.uint64))
    assert u[0] == 0.5 * 2.0**-32 and u[1] == 1 - 0.5 * 2.0**-32
    assert np.all((u > 0) & (u < 1))


def test_box_muller_closed_form():
    # u_b = 1/4 puts the angle at pi/2: first normal ~0, second = sqrt(-2 ln u_a)
    a, b = P.box_muller(np.array([np.exp(-0.5)]), np.array([0.25]))
    assert abs(a[0]) < 1e-15 and abs(b[0] - 1.0) < 1e-15


def test_site_normals_statistics():
    site = np.arange(100_000, dtype=np.uint64)
    N = P.site_normals(6, site, 17, 0, 3, 99)
    assert N.shape == (6, 100_000)
    for x in N:
        assert abs(x.mean()) < 5 / np.sqrt(x.size)
        assert abs(x.var() - 1) < 5 * np.sqrt(2 / x.size)
        assert stats.kstest(x, "norm").pvalue > 1e-4
    C = np.corrcoef(N)
    assert np.abs(C - np.eye(6)).max() < 0.02


def test_pair_normals_use_each_word_of_three_calls_once():
    # sites 2q and 2q + 1 share counter index q; calls 0..2 give W0..W11; site 2q + h
    # takes W_{6h}..W_{6h+5}: rebuilt here word by word from the generator itself
    q = np.array([0, 7, 12345, 2**31 - 1], dtype=np.uint64)
    step, stream, seed = 77, 5, 2**40 + 3
    W = []
    for call in range(3):
        W.extend(P.philox4x32_10(q, step, call, stream, seed))
    for h in (0, 1):
        N = P.pair_normals(2 * q + h, step, 0, stream, seed)
        for m in range(3):
            a, b = P.box_muller(P.uniform_fp64(W[6 * h + 2 * m]), P.uniform_fp64(W[6 * h + 2 * m + 1]))
            assert np.array_equal(N[2 * m], a) and np.array_equal(N[2 * m + 1], b)
    # the first site of a pair draws exactly what site_normals draws for the index q
    assert np.array_equal(P.pair_normals(2 * q, step, 0, stream, seed), P.site_normals(6, q, step, 0, stream, seed))


def test_pair_normals_statistics():
    # twelve normals of a site pair: unit normal, mutually uncorrelated, and independent
    # of the neighbouring pair's
    site = np.arange(200_000, dtype=np.uint64)
    N = P.pair_normals(site, 17, 0, 3, 99)
    assert N.shape == (6, 200_000)
    for x in N:
        assert abs(x.mean()) < 5 / np.sqrt(x.size)
        assert abs(x.var() - 1) < 5 * np.sqrt(2 / x.size)
        assert stats.kstest(x, "norm").pvalue > 1e-4
    both = np.concatenate([N[:, 0::2], N[:, 1::2]])          # (12, pairs): even site, odd site
    C = np.corrcoef(both)
    assert np.abs(C - np.eye(12)).max() < 0.02
    nxt = np.concatenate([N[:, 0:-2:2], N[:, 2::2]])         # pair q against pair q + 1
    assert np.abs(np.corrcoef(nxt) - np.eye(12)).max() < 0.02
