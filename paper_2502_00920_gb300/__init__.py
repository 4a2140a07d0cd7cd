"""GB300-native moment-chain lattice Boltzmann method for non-linear solids.

The compute path is the CUDA library ``liblbs.so`` (sm_103a) behind the C ABI
declared in ``include/lbs.h``; ``paper_2502_00920_gb300.lbs`` is its ctypes
binding.  ``paper_2502_00920_gb300.inputs`` holds the seeded workloads.

Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["inputs", "lbs"]
