"""CPU FP64 oracle for the moment-chain LBM (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg import this package.  The product path never does.
"""
from .oracle import OracleSim, build, lib, params, first_piola, pi_of_h, equilibrium, forcing, gradient, load  # noqa: F401
