"""Lattice tables of the oracle (test infrastructure only, see ``oracle/__init__``).

D2Q9: velocity set and moment matrix m_i^a exactly as printed in Sec. 3 (Eq. 9).
The printed weight list has only eight entries for nine velocities; the oracle
takes w = (4/9, 1/9 x4, 1/36 x4), the standard D2Q9 weights and the only choice
for which the printed m_i^a satisfy the Hermite orthonormality of Eq. 4
(pinned in tests/test_oracle_tables.py).

D1Q3: the paper reports D1Q3 results without printing its matrix (Sec. 3).
The oracle builds it as the projection of D2Q9 onto one axis: v = (0, +1, -1),
w = (2/3, 1/6, 1/6) and the Hermite polynomials 1, sqrt(3) v, (3 v^2 - 1)/sqrt(2)
normalised in the w-weighted norm of Eq. 4.

Moment roles (Sec. 3, after Eq. 9): a = 0 density, a = 1, 2 momentum (times
sqrt 3), a = 3, 4 shear stress, a = 5 bulk stress, a = 6, 7, 8 ghost moments.
D1Q3: a = 0 density, a = 1 momentum (times sqrt 3), a = 2 the single stress mode.

Parity: pinned (orthonormality, completeness, equilibrium-moment closed forms of
Eq. 10, D1Q3 = projection of D2Q9).
"""
import numpy as np

_S3 = np.sqrt(3.0)
_S32 = np.sqrt(1.5)
_S6 = np.sqrt(6.0)


class Lattice:
    """Velocities v[i, d], weights w[i], moment matrix m[a, i], back transform n[i, a]."""

    def __init__(self, name, v, w, m, conserved):
        self.name = name
        self.v = np.asarray(v, dtype=np.float64)          # (q, d)
        self.w = np.asarray(w, dtype=np.float64)          # (q,)
        self.m = np.asarray(m, dtype=np.float64)          # (q moments, q populations)
        self.n = (self.w[:, None] * self.m.T).copy()      # n_i^a = w_i m_i^a  (Sec. 2)
        self.q, self.d = self.v.shape
        self.conserved = tuple(conserved)                  # density and momentum moments
        self.nonconserved = tuple(a for a in range(self.q) if a not in self.conserved)


# Sec. 3: velocity order (0,0), (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1).
D2Q9 = Lattice(
    "D2Q9",
    v=[(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)],
    w=[4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36],
    # Eq. 9, row by row (moment a), column by column (population i).
    m=[
        [1, 1, 1, 1, 1, 1, 1, 1, 1],
        [0, _S3, 0, -_S3, 0, _S3, -_S3, -_S3, _S3],
        [0, 0, _S3, 0, -_S3, _S3, _S3, -_S3, -_S3],
        [0, 1.5, -1.5, 1.5, -1.5, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 3, -3, 3, -3],
        [-1, 0.5, 0.5, 0.5, 0.5, 2, 2, 2, 2],
        [0, -_S32, 0, _S32, 0, _S6, -_S6, -_S6, _S6],
        [0, 0, -_S32, 0, _S32, _S6, _S6, -_S6, -_S6],
        [0.5, -1, -1, -1, -1, 2, 2, 2, 2],
    ],
    conserved=(0, 1, 2),
)

_v1 = np.array([0.0, 1.0, -1.0])
D1Q3 = Lattice(
    "D1Q3",
    v=_v1[:, None],
    w=[2 / 3, 1 / 6, 1 / 6],
    m=[np.ones(3), _S3 * _v1, (3 * _v1**2 - 1) / np.sqrt(2.0)],
    conserved=(0, 1),
)

LATTICES = {"D1Q3": D1Q3, "D2Q9": D2Q9}


def equilibrium(lat, rho, u):
    """Local equilibrium f_i^0 of Eq. 2 with c = 1.

    rho: array of shape S; u: array of shape (d,) + S.  Returns (q,) + S.
    """
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    uv = np.tensordot(lat.v, u, axes=(1, 0))               # (q,) + S : u . v_i
    uu = np.sum(u * u, axis=0)                             # S : u . u
    w = lat.w.reshape((lat.q,) + (1,) * rho.ndim)
    return rho * w * (1.0 + 3.0 * uv + 4.5 * uv**2 - 1.5 * uu)
