"""Seeded synthetic workloads shared by the tests, the bench and the oracle runs.

This package holds input data only (lattice and direction matrices, coset shifts, array shapes,
seeded random points and coefficients, the closed-form test signal).  It contains none of the
method's arithmetic and imports neither the oracle nor the CUDA product path.
"""
from .workloads import *  # noqa: F401,F403
