"""CPU FP64 oracle for the lattice convolution sum (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of ``bench.py`` may
import this package.  It shares no code with the CUDA product path.
"""
from .oracle import (  # noqa: F401
    Spline, VoronoiSpline, build, lattice_sites, eval_sum, adjoint, cells, folded_offsets, zonotope_tiles,
    prefilter, d4_quasi_interpolation_taps,
)
