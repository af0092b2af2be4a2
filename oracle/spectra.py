"""Structure factors and cross correlators of the oracle (test infrastructure only).

Sec. 3, Eq. 11: dX(k) = sum_x dX(x) exp(-i k.x) over all lattice sites, with
k = 2 pi (kx / nx, ky / ny); the normalised static structure factor is
S_k(X) = N^X < dX(k) dX(-k) >, and Eq. 12 gives the cross correlator
R_k(X, Y) = N^X < X(k) Y(k)^* >.  For real fields dX(-k) = dX(k)^*, so both are
the one form C_ab(k) = N^{ab} < X_a(k) X_b(k)^* >.

Readings:
* Normalisation (Sec. 3 prints N^rho = 1/(rho^3 V), N^u = 1/(rho V k_B T) in
  units where they make the theory value 1 at rho0 = 1): the oracle uses the
  per-field variances of Eq. 7, N^{M^a} = 1 / (V mu rho0) for every moment
  (density included, mu = 3 k_B T) and N^{u} = rho0 / (V k_B T) for velocity
  components, and the geometric mean sqrt(N^a N^b) for a pair.  These equal the
  printed values at rho0 = 1, k_B T = 1/3.
* delta M = M - <M>: at k = 0 the product of the sampled means is subtracted;
  at k != 0 the mean does not contribute.

Parity: the DFT is pinned against numpy.fft.fft2 and Parseval; normalisation
against the theory value 1 of Eq. 7 (tests/test_oracle_stats.py).
"""
import numpy as np


def dft2(x):
    """Separable direct DFT, X(ky, kx) = sum_{y,x} x(y, x) exp(-2 pi i (kx x/nx + ky y/ny))."""
    ny, nx = x.shape
    ex = np.exp(-2j * np.pi * np.outer(np.arange(nx), np.arange(nx)) / nx)
    ey = np.exp(-2j * np.pi * np.outer(np.arange(ny), np.arange(ny)) / ny)
    return ey @ (x.astype(np.complex128) @ ex)


def field_variance(p, fid):
    """Per-site equal-time variance of a field in the ideal gas (Eq. 7 with mu = 3 k_B T)."""
    if fid < p.lat.q:
        return p.mu * p.rho0
    return p.kT / p.rho0


def pairs(fields):
    fs = list(fields)
    return [(fs[i], fs[j]) for i in range(len(fs)) for j in range(i, len(fs))]


class Accumulator:
    """Sums of X_a(k) X_b(k)^* over samples, for every field pair a <= b."""

    def __init__(self, p):
        self.p = p
        self.fields = list(p.fields)
        self.n = 0
        self.sum = {}
        self.mean0 = {f: 0.0 for f in self.fields}

    def add(self, fields):
        X = {fid: dft2(np.asarray(v).reshape(self.p.ny if self.p.lat.d == 2 else 1, self.p.nx))
             for fid, v in fields.items()}
        for a, b in pairs(self.fields):
            prod = X[a] * np.conj(X[b])
            self.sum[(a, b)] = self.sum.get((a, b), 0.0) + prod
        for fid in self.fields:
            self.mean0[fid] += X[fid][0, 0]
        self.n += 1

    def correlator(self, a, b):
        """Normalised C_ab(k) on the full (ny, nx) grid, complex."""
        p = self.p
        key = (a, b) if (a, b) in self.sum else (b, a)
        c = self.sum[key] / self.n
        if key != (a, b):
            c = np.conj(c)
        c = c.copy()
        c[0, 0] -= (self.mean0[a] / self.n) * np.conj(self.mean0[b] / self.n)
        V = p.nx * (p.ny if p.lat.d == 2 else 1)
        norm = 1.0 / (V * np.sqrt(field_variance(p, a) * field_variance(p, b)))
        return c * norm


def dft_at(x, kx, ky):
    """X(k) for one wave vector by the direct sum over all sites (large lattices)."""
    ny, nx = x.shape
    ex = np.exp(-2j * np.pi * kx * np.arange(nx) / nx)
    ey = np.exp(-2j * np.pi * ky * np.arange(ny) / ny)
    return ey @ (x.astype(np.complex128) @ ex)


class PointAccumulator:
    """Accumulator restricted to a list of wave vectors (ky, kx), same normalisation."""

    def __init__(self, p, kpoints):
        self.p = p
        self.fields = list(p.fields)
        self.k = list(kpoints)
        self.n = 0
        self.X = []

    def add(self, fields):
        ny = self.p.ny if self.p.lat.d == 2 else 1
        X = {fid: np.array([dft_at(np.asarray(v).reshape(ny, self.p.nx), kx, ky) for ky, kx in self.k])
             for fid, v in fields.items()}
        X0 = {fid: float(np.sum(v)) for fid, v in fields.items()}
        self.X.append((X, X0))
        self.n += 1

    def correlator(self, a, b):
        p = self.p
        c = sum(X[a] * np.conj(X[b]) for X, _ in self.X) / self.n
        m_a = sum(X0[a] for _, X0 in self.X) / self.n
        m_b = sum(X0[b] for _, X0 in self.X) / self.n
        c = c.copy()
        for i, (ky, kx) in enumerate(self.k):
            if kx == 0 and ky == 0:
                c[i] -= m_a * m_b
        V = p.nx * (p.ny if p.lat.d == 2 else 1)
        return c / (V * np.sqrt(field_variance(p, a) * field_variance(p, b)))


class TimeAccumulator:
    """Time correlators at a list of wave vectors (an extension the paper leaves to
    future work, Sec. 3: its correlators are equal-time ones).

    For samples s = 0, 1, ... (every sample_every steps) and lag tau = 0 .. n_lags - 1
    (in samples), with every ordered field pair (a, b):

        F_ab(k, tau) = N^{ab} (1 / n_tau) sum_{s >= tau} X_a(k, s) X_b(k, s - tau)^*,

    n_tau = n - tau pairs of samples, N^{ab} the normalisation of the equal-time
    correlators (so F_ab(k, 0) = C_ab(k) away from k = 0; k = 0 is not allowed, there
    the mean would have to be removed).  X(k) is the direct sum of Eq. 11.
    """

    def __init__(self, p, kpoints, n_lags):
        self.p = p
        self.fields = list(p.fields)
        self.k = [tuple(k) for k in kpoints]
        if any(kx == 0 and ky == 0 for ky, kx in self.k):
            raise ValueError("k = 0 is not supported")
        self.T = int(n_lags)
        self.hist = []                                   # last T samples: {fid: (n_k,) complex}
        self.n = 0
        self.sum = {(a, b): np.zeros((self.T, len(self.k)), complex) for a in self.fields for b in self.fields}

    def add(self, fields):
        ny = self.p.ny if self.p.lat.d == 2 else 1
        X = {fid: np.array([dft_at(np.asarray(v).reshape(ny, self.p.nx), kx, ky) for ky, kx in self.k])
             for fid, v in fields.items()}
        self.hist.insert(0, X)                           # hist[tau] = sample s - tau
        del self.hist[self.T:]
        for (a, b), acc in self.sum.items():
            for tau, Y in enumerate(self.hist):
                acc[tau] += X[a] * np.conj(Y[b])
        self.n += 1

    def correlator(self, a, b):
        """Normalised F_ab(k, tau), shape (n_lags, n_k); lags without pairs are NaN."""
        p = self.p
        V = p.nx * (p.ny if p.lat.d == 2 else 1)
        norm = 1.0 / (V * np.sqrt(field_variance(p, a) * field_variance(p, b)))
        n_tau = np.array([self.n - t for t in range(self.T)], float)
        with np.errstate(invalid="ignore", divide="ignore"):
            return np.where(n_tau[:, None] > 0, self.sum[(a, b)] / n_tau[:, None], np.nan) * norm
