"""B300-native evaluator of the lattice convolution sum f(x) = sum_n c_n phi(x - n) for box splines
on Cartesian, BCC, FCC and D4* lattices (Horacsek & Alim, arXiv 2102.08514).

    gen/       host-side exact-rational generator (pieces, stencils, polynomial tables)
    csrc/      sm_103a CUDA kernels and the C ABI (include/interp.h)
    binding.py thin ctypes binding with the C names, plus Interpolator / lattice_interp
    build.py   in-tree nvcc build of libinterp_b300.so
"""
import importlib

__all__ = ["Interpolator", "lattice_interp"]


def __getattr__(name):
    if name in ("Interpolator", "lattice_interp"):
        return getattr(importlib.import_module(".binding", __name__), name)
    raise AttributeError(name)
