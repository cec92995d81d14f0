"""Helpers shared by the GPU parity tests (test code only)."""
import json
import os
from fractions import Fraction

import numpy as np

from synth import LATTICES, SPLINES, interior_box, make_rng, uniform_points

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLES_JSON = os.path.join(ROOT, "paper_2102_08514_b300", "csrc", "generated", "splines.json")

# value tolerance of the benchmark spec: max-abs error <= 2e-6 * max|c|
VALUE_TOL = 2e-6


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def spline_setup(name):
    sp = SPLINES[name]
    lat = LATTICES[sp.lattice]
    xi = np.asarray(sp.xi)
    detl = abs(round(np.linalg.det(np.asarray(lat.L, dtype=float))))
    return sp, lat, xi, detl


class OracleSpline:
    """The oracle's basis for a built-in spline name: oracle.Spline for a box spline,
    oracle.VoronoiSpline for a Voronoi spline (generators = xi / 2), one interface."""

    def __init__(self, name):
        import oracle
        sp, lat, xi, detl = spline_setup(name)
        if sp.order:
            gens = [tuple(Fraction(int(v), 2) for v in col) for col in xi.T]
            self.v, self.sp = oracle.VoronoiSpline(lat.L, gens, sp.order), None
        else:
            self.v, self.sp = None, oracle.Spline(xi, detl)
        self.halfwidth = (self.v or self.sp).halfwidth

    def phi(self, z, grad=False):
        return (self.v or self.sp).phi(z, grad=grad)

    def eval_sum(self, D, cosets, c, pts, grad=False):
        import oracle
        c = np.asarray(c, dtype=np.float64)
        pts = np.asarray(pts, dtype=np.float64)
        if self.v is not None:
            return self.v.eval_sum(D, cosets, c, pts, grad=grad)
        return oracle.eval_sum(self.sp, D, cosets, c, pts, grad=grad)

    def adjoint(self, D, cosets, shape, pts, g):
        import oracle
        pts = np.asarray(pts, dtype=np.float64)
        g = np.asarray(g, dtype=np.float64)
        if self.v is not None:
            return self.v.adjoint(D, cosets, shape, pts, g)
        return oracle.adjoint(self.sp, D, cosets, shape, pts, g)


def make_interpolator(name, dims, storage="f32"):
    """The CUDA path's handle: by (L, Xi) for a box spline, by name for a Voronoi spline."""
    from paper_2102_08514_b300.binding import Interpolator
    sp, lat, xi, detl = spline_setup(name)
    if sp.order:
        return Interpolator.named(name, dims, storage)
    return Interpolator(np.asarray(lat.L), xi, dims, storage)


def mixed_points(name, dims, n, seed, outside=True):
    """Seeded FP32 points: mostly uniform in the interior box, plus (if outside) points in a band
    around the data (zero-extension region), exact ties on cell boundaries and far-away points."""
    lo, hi = interior_box(name, dims)
    rng = make_rng(seed, 11)
    n_in = n if not outside else (n * 3) // 4
    pts = [uniform_points(rng, n_in, lo, hi)]
    if outside:
        lat = LATTICES[SPLINES[name].lattice]
        ext_lo = -2.0 * lat.D - 1.0
        ext_hi = lat.D * np.asarray(dims) + 1.0
        m = n - n_in
        band = uniform_points(rng, m - m // 4, np.full(len(dims), ext_lo), ext_hi)
        ties = np.round(uniform_points(rng, m // 4, lo, hi) * 2.0) / 2.0      # integers and halves
        pts += [band, ties.astype(np.float32)]
    return np.concatenate(pts, axis=0).astype(np.float32)


def tables():
    with open(TABLES_JSON) as f:
        return json.load(f)["splines"]


def grad_bound(name, pts):
    """G = max over pts of sum_n |grad phi(x - n)|_inf, from the oracle (at least 1)."""
    import oracle
    sp, lat, xi, detl = spline_setup(name)
    o = OracleSpline(name)
    G = 1.0
    for x in np.asarray(pts, dtype=np.float64):
        sites = oracle.lattice_sites(lat.L, x - o.halfwidth - 1, x + o.halfwidth + 1)
        _, g = o.phi(x - sites, grad=True)
        G = max(G, float(np.abs(g).max(axis=1).sum()))
    return G
