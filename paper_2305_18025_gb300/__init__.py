"""GB300-native bosonic PIMD exchange potential and forces.

Implements the hot path of Feldman & Hirshberg, "Quadratic Scaling Bosonic
Path Integral Molecular Dynamics": the exchange potential V^{[1,N]} of N ring
polymers with P beads and the force on every bead (Algorithm 1), as
hand-written sm_103a CUDA kernels behind the C ABI of ``include/bpimd.h``.

Modules
-------
``bpimd``     ctypes binding with the C ABI's names (argument marshalling only).
``exchange``  torch-facing wrappers: ``ExchangeEnergy`` (context + tensors), the
              autograd function whose backward is the force kernel, and
              ``RingPolymerMD`` (BAOAB Langevin steps of bpimd_step).
``inputs``    seeded synthetic inputs (no arithmetic of the method).
``build``     in-tree nvcc build of ``libbpimd.so``.

Importing the package does not load CUDA; the library is loaded on first use
and raises if it cannot be built or loaded (there is no CPU fallback).
"""

__all__ = ["bpimd", "exchange", "inputs", "build"]
