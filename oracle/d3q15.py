"""The D3Q15 view of the three-dimensional oracle (test infrastructure only).

The paper reports that it also tested D3Q15 (Sec. 3) without printing its tables; the
lattice, its Gram-Schmidt moment basis in the Eq. 4 norm and the step are defined in
``oracle.lb3d``, which this module re-exports with the D3Q15 lattice as ``LATTICE``
(``Params3`` defaults to it).

Parity: pinned in ``tests/test_oracle_lb3d.py`` (see ``oracle.lb3d``).
"""
from .lb3d import (LATTICES, V15 as V, W15 as W, Params3, PointAccumulator3, Run3, collide, dft_at,  # noqa: F401
                   macroscopic, point_theory, sample_fields, site_index, stream, thermal_state, uniform_state)

LATTICE = LATTICES["D3Q15"]
