"""Local-density noise amplitude (noise_mode 2): Eq. 8 with the site's own density
in place of rho-bar (oracle, CPU only)."""
import numpy as np

from oracle import lb, spectra, theory
from paper_1010_1233_gb300 import workloads as W
from test_oracle_stats import _batch_spectra, _check


def test_uniform_density_equals_the_global_form():
    kw = dict(lattice="D2Q9", nx=16, ny=8, tau=W.taus_d2q9(0.8, 0.7, 1.2), kT=1e-3, u0=(0.1, 0.0), seed=2)
    p0, p2 = lb.Params(**W.replica(**kw)), lb.Params(**W.replica(noise_mode=2, **kw))
    f = lb.uniform_state(p0)
    assert np.abs(lb.collide(p0, f, 3) - lb.collide(p2, f, 3)).max() < 1e-15


def test_noise_variance_follows_the_local_density():
    # two density plateaus 1.2 rho0 and 0.8 rho0: the sampled noise variances of every
    # non-conserved moment stand in the ratio 1.2 / 0.8 (within sampling error)
    p = lb.Params(**W.replica("D2Q9", 32, 32, W.taus_d2q9(0.8), kT=1e-4, seed=4, noise_mode=2))
    lat = p.lat
    f = lb.uniform_state(p)
    f[:, :16, :] *= 1.2
    f[:, 16:, :] *= 0.8
    hi, lo = [], []
    for t in range(16):
        _, parts = lb.collide(p, f, t, return_parts=True)
        xi = parts["xi"][list(lat.nonconserved)]
        hi.append(xi[:, :16, :].reshape(6, -1))
        lo.append(xi[:, 16:, :].reshape(6, -1))
    vh, vl = np.var(np.concatenate(hi, 1), axis=1), np.var(np.concatenate(lo, 1), axis=1)
    n = 16 * 16 * 32
    ratio = vh / vl
    assert np.all(np.abs(ratio - 1.5) < 5 * 1.5 * np.sqrt(4.0 / n)), ratio
    # and the global form does not see the plateaus
    p0 = lb.Params(**W.replica("D2Q9", 32, 32, W.taus_d2q9(0.8), kT=1e-4, seed=4))
    _, parts = lb.collide(p0, f, 0, return_parts=True)
    xi = parts["xi"][list(lat.nonconserved)]
    assert abs(np.var(xi[:, :16]) / np.var(xi[:, 16:]) - 1.0) < 0.1


def test_linear_statistics_unchanged():
    # the density factor multiplies the noise by 1 + O(drho): second order in the
    # fluctuations, so the linear theory of Eq. 8 still predicts the spectra
    p = lb.Params(**W.replica(nx=8, ny=8, tau=W.taus_d2q9(0.8, 0.8, 1.0), kT=1e-4, seed=3, u0=(0.1, 0.0),
                              init_mode=1, fields=[0, 9, 10], noise_mode=2))
    meas = _batch_spectra(p, 10, 600, warmup=300)
    _check(p, meas)
