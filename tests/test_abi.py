"""The C-ABI library loads, exports every declared symbol and validates its input (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1010_1233_gb300 import _lib as L, build, workloads as W
from paper_1010_1233_gb300.sim import replica_struct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return L.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(flb_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "flb_run" in names and "flb_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(L.exported_symbols()) | set(names)


def _ws(reps, precision=L.FLB_FP32_DEV):
    arr = (L.flb_replica * len(reps))(*[replica_struct(p) for p in reps])
    n = ctypes.c_size_t()
    rc = L.lib().flb_workspace_bytes(precision, arr, len(reps), ctypes.byref(n))
    return rc, n.value


def test_workspace_size_grows_with_lattice(lib):
    rc1, a = _ws([W.replica(nx=64, ny=64)])
    rc2, b = _ws([W.replica(nx=128, ny=64)])
    assert rc1 == rc2 == 0 and b > a >= 2 * 9 * 64 * 64 * 4
    rc3, c = _ws([W.replica(nx=64, ny=64, fields=(0, 9, 10))])
    assert rc3 == 0 and c > a


@pytest.mark.parametrize("bad", [
    dict(tau=W.taus_d2q9(0.5)),                     # tau must exceed 1/2
    dict(nx=7),                                     # odd nx
    dict(rho0=0.0),
    dict(noise_mask=1),                             # noise on density
    dict(fields=(0,), nx=24),                       # sampling needs powers of two
    dict(fields=(11,)),                             # unknown field
    dict(init_mode=3),
    dict(noise_mode=3),                             # unknown noise mode
    dict(nx=65536, ny=65536),                       # 2^32 sites
])
def test_invalid_parameters_rejected(lib, bad):
    p = W.replica(nx=16, ny=16)
    p.update(bad)
    rc, _ = _ws([p])
    assert rc == L.FLB_EINVAL
    assert len(lib.flb_last_error()) > 0


def test_mixed_lattices_rejected(lib):
    rc, _ = _ws([W.replica(nx=16, ny=16), W.replica("D1Q3", 16, 1, W.taus_d1q3(0.8))])
    assert rc == L.FLB_EINVAL


def test_d1q3_needs_single_row(lib):
    p = W.replica("D1Q3", 16, 1, W.taus_d1q3(0.8))
    p["ny"] = 4
    s = replica_struct(p)
    s.ny = 4
    arr = (L.flb_replica * 1)(s)
    n = ctypes.c_size_t()
    assert lib.flb_workspace_bytes(L.FLB_FP64, arr, 1, ctypes.byref(n)) == L.FLB_EINVAL


def test_empty_replica_list_rejected(lib):
    n = ctypes.c_size_t()
    assert lib.flb_workspace_bytes(L.FLB_FP32_DEV, None, 0, ctypes.byref(n)) == L.FLB_EINVAL


def test_d3q15_workspace(lib):
    rc, a = _ws([W.replica3(16, 8, 4)])
    assert rc == 0 and a >= 2 * 15 * 16 * 8 * 4 * 4
    rc, b = _ws([W.replica3(16, 8, 4, fields=(0, 4, 14))])
    assert rc == 0 and b >= a + 3 * 16 * 8 * 4 * 4
    rc, c = _ws([W.replica3(16, 8, 4)], precision=L.FLB_FP64)
    assert rc == 0 and c >= 2 * 15 * 16 * 8 * 4 * 8


@pytest.mark.parametrize("bad", [
    dict(nz=0),                                     # D3Q15 needs nz >= 1
    dict(nx=5),                                     # odd nx
    dict(tau=W.taus_d3q15(0.5)),                    # tau must exceed 1/2
    dict(noise_mask=1 << 3),                        # noise on momentum z
    dict(noise_mask=1 << 15),                       # beyond moment 14
    dict(fields=(15,)),                             # unknown field
    dict(fields=tuple(range(12))),                  # more than 11 fields
    dict(noise_mode=1),                             # mode 0 only
    dict(nx=4096, ny=4096, nz=256),                 # 2^32 sites
    dict(nx=8192, ny=2, nz=2, fields=(0,)),         # direct transforms: nx <= 4096
])
def test_invalid_d3q15_parameters_rejected(lib, bad):
    p = W.replica3(8, 8, 8)
    p.update(bad)
    rc, _ = _ws([p])
    assert rc == L.FLB_EINVAL
    assert len(lib.flb_last_error()) > 0


def test_nz_rejected_on_2d_lattices(lib):
    s = replica_struct(W.replica(nx=16, ny=16))
    s.nz = 2
    arr = (L.flb_replica * 1)(s)
    n = ctypes.c_size_t()
    assert lib.flb_workspace_bytes(L.FLB_FP32_DEV, arr, 1, ctypes.byref(n)) == L.FLB_EINVAL


def test_d3q19_workspace_and_validation(lib):
    rc, a = _ws([W.replica3(16, 8, 4, lattice="D3Q19")])
    assert rc == 0 and a >= 2 * 19 * 16 * 8 * 4 * 4
    for bad in (dict(fields=(19,)), dict(noise_mask=1 << 19), dict(noise_mask=1 << 2), dict(nz=0),
                dict(tau=W.taus_d3q19(0.5))):
        p = W.replica3(8, 8, 8, lattice="D3Q19")
        p.update(bad)
        rc, _ = _ws([p])
        assert rc == L.FLB_EINVAL, bad
    rc, _ = _ws([W.replica3(8, 8, 8, lattice="D3Q19", fields=(18,))])
    assert rc == 0
    rc, _ = _ws([W.replica3(8, 8, 8), W.replica3(8, 8, 8, lattice="D3Q19")])       # mixed lattices
    assert rc == L.FLB_EINVAL


def test_bounds_counters_only_in_the_checked_build(lib):
    # the normal build carries no index checks: the counter query answers FLB_ESTATE
    # without touching the device; NULL arguments are rejected first
    n, site = ctypes.c_uint64(7), ctypes.c_uint32(7)
    assert lib.flb_debug_bounds(None, ctypes.byref(site), 0) == L.FLB_EINVAL
    assert lib.flb_debug_bounds(ctypes.byref(n), ctypes.byref(site), 1) == L.FLB_ESTATE
    assert n.value == 0 and site.value == 0
    assert b"--checked" in lib.flb_last_error()


def test_kernel_launch_query_validates(lib):
    # the launch count is read from the context; NULL arguments are rejected on the host
    n = ctypes.c_uint64(5)
    assert lib.flb_kernel_launches(None, ctypes.byref(n)) == L.FLB_EINVAL
    assert n.value == 5


def test_bench_workload_workspace(lib):
    # HBM layout of the 16384^2 D2Q9 workload (FP32 deviations, rho/u_x/u_y sampled):
    # two population buffers, the fields, two spectrum slots (two samples folded into one
    # accumulation pass) in the column-tiled layout [F][ceil((nx/2+1)/16)][ny][16], and the
    # FP64 pair sums (3 autos x 8 B + 3 cross pairs x 16 B per k point) over the half
    # spectrum padded to the 8-column accumulation tiles; the rest (descriptors, twiddle
    # tables, k = 0 sums, alignment) stays below 1 MB.  38.7 GB of the GPU's 288.
    N, F = 16384, 3
    p = W.d2q9_16384(N)["replicas"][0]
    rc, n = _ws([p])
    pops, fields = 2 * 9 * 4 * N * N, F * 4 * N * N
    spec_slot = F * -(-(N // 2 + 1) // 16) * N * 16 * 8
    sums = 72 * N * (-(-(N // 2 + 1) // 8) * 8)
    assert rc == 0
    assert 0 <= n - (pops + fields + 2 * spec_slot + sums) < 1 << 20, n
    q = dict(p, fields=())
    rc, m = _ws([q])
    assert rc == 0 and 0 <= m - pops < 1 << 20, m                  # no sampling: populations only
