"""Plain FP64 CPU oracle for fluctuating ideal-gas lattice Boltzmann with ghost noise.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  It shares no code, table or constant with the CUDA
library in ``paper_1010_1233_gb300/``; both sides only share the seeded input
generators in ``paper_1010_1233_gb300/workloads.py`` (which hold none of the
method's arithmetic).

The method is the one analysed in Kaehler & Wagner, "Cross Correlators and
Galilean Invariance in Fluctuating Ideal Gas Lattice Boltzmann Simulations":

* ``lattice``  -- D2Q9 (Sec. 3, Eq. 9) and D1Q3 velocity sets, weights and the
  Hermite-orthonormal moment matrix m_i^a (Eq. 4), back transform n_i^a = w_i m_i^a.
* ``philox``   -- counter-based Philox4x32-10 (Salmon et al., SC'11) and the
  Box-Muller map to the unit-variance N of Eq. 8.
* ``lb``       -- the step of Eq. 1 / Eq. 5 in dense f-space: pull-stream,
  moments (Eq. 3), equilibrium (Eq. 2), relaxation of non-conserved moments,
  noise (Eq. 8) on stress and ghost moments, back transform.
* ``spectra``  -- direct separable DFT and the structure factors / cross
  correlators of Eqs. 11-12.
* ``theory``   -- exact stationary covariance of the linearised dynamics
  (discrete Lyapunov equation per wave vector), which reduces to Eq. 7 at u0 = 0.
* ``mlp``      -- FP64 forward/backward of the per-site noise-scale network and
  of its correlator loss (not in the paper; a learned extension).
* ``lb3d``     -- the same scheme on the three-dimensional D3Q15 (which Sec. 3 reports
  testing) and D3Q19 lattices: Gram-Schmidt moment bases in the Eq. 4 norm, step,
  thermal start, direct DFT at chosen wave vectors, linear theory per k
  (``d3q15`` is its D3Q15 view).

Parity status per function is stated in each module header.
"""
