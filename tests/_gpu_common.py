"""Helpers shared by the GPU parity tests (test code only)."""
import json
import os

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
    o = oracle.Spline(xi, detl)
    G = 1.0
    for x in np.asarray(pts, dtype=np.float64):
        sites = oracle.lattice_sites(lat.L, x - o.halfwidth - 1, x + o.halfwidth + 1)
        _, g = o.phi(x - sites, grad=True)
        G = max(G, float(np.abs(g).max(axis=1).sum()))
    return G
