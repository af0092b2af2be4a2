"""GB300-native fluctuating ideal-gas lattice Boltzmann with ghost noise.

The method of Kaehler & Wagner, "Cross Correlators and Galilean Invariance in
Fluctuating Ideal Gas Lattice Boltzmann Simulations": D1Q3/D2Q9 (and the 3D
D3Q15/D3Q19) lattice Boltzmann with Hermite-orthonormal moments,
fluctuation-dissipation noise on every non-conserved moment, and equal-time
structure factors / cross correlators (and time correlators at chosen wave
vectors).  The compute path is libflb.so (hand-written sm_103a CUDA behind
the C ABI of include/flb.h); this package binds it.
"""
from .sim import Sim, philox, replica_struct, bf16_bits, stability  # noqa: F401
from . import workloads  # noqa: F401
