"""The product path has no CPU fallback: without the compiled library, or without a CUDA
device, the binding raises instead of computing anything on the host."""
import os

import pytest
import torch

from paper_1010_1233_gb300 import _lib as L, Sim, workloads as W


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", os.path.join(os.path.dirname(L.LIB_PATH), "no_such_libflb.so"))
    with pytest.raises(RuntimeError, match="missing"):
        L.lib()


@pytest.mark.skipif(torch.cuda.is_available(), reason="the behaviour without a CUDA device")
def test_simulation_without_cuda_device_raises():
    p = W.replica("D2Q9", 16, 16, W.taus_d2q9(0.8), kT=1e-4, seed=1)
    with pytest.raises((RuntimeError, AssertionError, L.FlbError)):
        Sim(p, precision="fp32")
