"""flb_spectra_accumulate (caller-provided fields and scratch) against the oracle's sums (GPU)."""
import numpy as np
import pytest
import torch

from oracle import lb, spectra
from paper_1010_1233_gb300 import workloads as W
from paper_1010_1233_gb300.sim import spectra_accumulate, unpack_pair_sums

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,F,ny,nx,tol", [
    ("fp64", 3, 16, 32, 1e-12), ("fp64", 4, 2048, 8, 1e-12),      # one-pass / four-step columns
    ("fp32", 5, 64, 128, 2e-6), ("fp32", 1, 8, 16384, 2e-6), ("fp32", 3, 4096, 8, 2e-6),
    # rows of the Stockham row pass: passes 16-16-8 (4096), 16-16-16-2 (8192), 16-16-16-4 (32768)
    ("fp32", 2, 4, 4096, 2e-6), ("fp32", 2, 4, 8192, 2e-6), ("fp32", 1, 2, 32768, 2e-6)])
def test_spectra_accumulate_matches_oracle(precision, F, ny, nx, tol):
    dt = torch.float64 if precision == "fp64" else torch.float32
    p = lb.Params(**W.replica(nx=nx, ny=ny, fields=list(range(F))))
    acc = spectra.Accumulator(p) if nx * ny <= 65536 else None
    sums = mean0 = None
    X_all = []
    for s in range(2):
        x = W.random_perturbation((F, ny, nx), 40 + s) + 0.3
        X_all.append(x)
        xt = torch.tensor(x, dtype=dt, device="cuda")
        sums, mean0 = spectra_accumulate(xt, sums, mean0)
    torch.cuda.synchronize()
    got = unpack_pair_sums(sums, F, ny, nx)
    m0 = mean0.cpu().numpy()
    xr = [np.asarray(torch.tensor(x, dtype=dt).double()) for x in X_all]   # inputs as the GPU saw them
    m0_tol = 1e-12 if precision == "fp64" else 1e-6          # FP32 transforms: ~log2(V) eps
    for a in range(F):
        assert abs(m0[a] - sum(x[a].sum() for x in xr)) < m0_tol * sum(np.abs(x[a]).sum() for x in xr)
    hn = nx // 2 + 1
    for (a, b), g in got.items():
        if nx * ny <= 65536:
            want = sum(spectra.dft2(x[a]) * np.conj(spectra.dft2(x[b])) for x in xr)[:, :hn]
        else:
            ks = [(0, 0), (1, 1), (ny - 1, hn - 1), (ny // 2, hn // 2), (3, min(5, hn - 1))]
            want = np.zeros((ny, hn), complex)
            for ky, kx in ks:
                want[ky, kx] = sum(spectra.dft_at(x[a], kx, ky) * np.conj(spectra.dft_at(x[b], kx, ky)) for x in xr)
            g = np.where(want != 0, g, 0)
        scale = max(np.abs(want).max(), 1.0)
        assert np.abs(g - want).max() < tol * scale * np.log2(nx * ny), (a, b)


def test_spectra_accumulate_rejects_bad_sizes():
    from paper_1010_1233_gb300 import _lib as L
    x = torch.zeros((2, 12, 16), device="cuda")
    with pytest.raises(L.FlbError):
        spectra_accumulate(x)
