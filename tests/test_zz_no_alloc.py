"""flb_spectra_accumulate_static: correlator sampling with no device allocation (GPU).

For callers that cannot allocate device memory (a framework that owns the
whole memory budget, a memory-capped service, a loop that must not pay for
cudaMalloc's synchronisation), this entry point keeps its scratch in a fixed
8 MiB device array inside the library.  This test calls it through the C ABI
and compares its sums with those of flb_spectra_accumulate (caller scratch) on
the same inputs, after each of two calls in a row, including a plan within 14 %
of the array's size; it checks that repeated calls leave the device's free
memory unchanged, and the size limit.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1010_1233_gb300 import _lib as L, build, workloads as W
from paper_1010_1233_gb300.sim import spectra_accumulate, spectra_sizes

pytestmark = pytest.mark.gpu

_PREC = {torch.float32: L.FLB_FP32_DEV, torch.float64: L.FLB_FP64}


def _static(lib, x, sums, mean0):
    F, ny, nx = x.shape
    return lib.flb_spectra_accumulate_static(
        _PREC[x.dtype], nx, ny, F, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(sums.data_ptr()),
        ctypes.c_void_p(mean0.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.fixture(scope="module")
def lib():
    build.build()
    lib = L.lib()
    f = lib.flb_spectra_accumulate_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return lib


# the last case's plan needs 7.2 MB, within 14 % of the 8 MiB array
@pytest.mark.parametrize("dtype,F,ny,nx,tol", [(torch.float32, 3, 128, 256, 2e-6),
                                               (torch.float64, 4, 2048, 8, 1e-12),
                                               (torch.float64, 11, 4096, 16, 1e-12)])
def test_static_scratch_matches_caller_scratch(lib, dtype, F, ny, nx, tol):
    _, ns = spectra_sizes(F, ny, nx, "fp64" if dtype == torch.float64 else "fp32")
    ref_sums = ref_m0 = None
    sums = torch.zeros(ns, dtype=torch.float64, device="cuda")
    m0 = torch.zeros(F, dtype=torch.float64, device="cuda")
    for call in range(2):
        x = torch.tensor(W.random_perturbation((F, ny, nx), 70 + call) + 0.2, dtype=dtype, device="cuda")
        ref_sums, ref_m0 = spectra_accumulate(x, ref_sums, ref_m0)
        assert _static(lib, x, sums, m0) == L.FLB_OK, lib.flb_last_error()
        torch.cuda.synchronize()
        scale = max(ref_sums.abs().max().item(), 1.0)
        assert (sums - ref_sums).abs().max().item() <= tol * scale * np.log2(nx * ny), call
        assert (m0 - ref_m0).abs().max().item() <= tol * max(ref_m0.abs().max().item(), 1.0), call


def test_static_scratch_rejects_oversize(lib):
    F, ny, nx = 11, 512, 512          # needs ~11.6 MB of scratch, above the 8 MiB array
    x = torch.zeros((F, ny, nx), dtype=torch.float32, device="cuda")
    sums = torch.zeros(1, dtype=torch.float64, device="cuda")
    m0 = torch.zeros(F, dtype=torch.float64, device="cuda")
    assert _static(lib, x, sums, m0) == L.FLB_EINVAL
    assert b"static array" in lib.flb_last_error()


def test_static_calls_allocate_nothing(lib):
    # after one call (which may load the library's module and with it the array), further
    # calls leave the device's free memory unchanged
    F, ny, nx = 3, 256, 256
    _, ns = spectra_sizes(F, ny, nx, "fp32")
    x = torch.tensor(W.random_perturbation((F, ny, nx), 91), dtype=torch.float32, device="cuda")
    sums = torch.zeros(ns, dtype=torch.float64, device="cuda")
    m0 = torch.zeros(F, dtype=torch.float64, device="cuda")
    assert _static(lib, x, sums, m0) == L.FLB_OK, lib.flb_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert _static(lib, x, sums, m0) == L.FLB_OK, lib.flb_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
