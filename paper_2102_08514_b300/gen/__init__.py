"""Host-side generator: exact rational analysis of a box spline (or of a Voronoi spline, a sum of
shifted box splines) on an integer lattice.

It splits the per-coset region of evaluation into polynomial pieces, folds it under the
symmetry group of the spline (signed permutations), and emits per-piece polynomial coefficient
tables and coefficient-gather stencils for the CUDA kernels (Sec. 4.1--4.3 of Horacsek & Alim,
arXiv 2102.08514).
"""
from .pieces import analyse, analyse_voronoi, SplineTables  # noqa: F401
from .catalog import CATALOG, VORONOI, catalog_entry  # noqa: F401
