"""Generator checks on the CPU (no GPU): the shipped tables against the oracle.

The tables in csrc/generated/splines.json (exact rationals) are evaluated here by a plain
table-driven evaluator written in this test -- shift to the nearest coset site, fold by the signed
permutation, plane sign bits, sigma, stencil gather, exact polynomial -- and compared with the
oracle's brute-force recurrence.  Also: the pieces tile the folded region, sigma names the piece
containing every point, the mean stencil size is Table 1's '# Lookups', and the committed header
matches a fresh run of the generator.
"""
import itertools
import json
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import oracle
from synth import LATTICES, SPLINES

from _gpu_common import OracleSpline

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEN = os.path.join(ROOT, "paper_2102_08514_b300", "csrc", "generated")
NAMES = ["bcc_linear", "bcc_quintic", "fcc_6dir", "cc_7dir", "d4s_8dir", "d4_8dir", "bcc_quartic", "cc_linear_rd", "cc_voronoi1",
         "cc_voronoi2", "cc_voronoi3", "bcc_voronoi1", "fcc_voronoi1", "fcc_voronoi2", "bcc_voronoi2"]
# Table 1 '# Lookups' (and Sec. 5.2 for D4*)
TABLE1_LOOKUPS = {"bcc_linear": 4, "bcc_quintic": 32, "fcc_6dir": 16, "cc_7dir": 53, "d4s_8dir": 60, "d4_8dir": 240,
                  "bcc_quartic": 30,
                  "cc_linear_rd": 16, "cc_voronoi1": 8, "cc_voronoi2": 27, "cc_voronoi3": 64, "bcc_voronoi1": 8,
                  "bcc_voronoi2": 27, "fcc_voronoi1": 8, "fcc_voronoi2": 27}


@pytest.fixture(scope="module")
def tables():
    with open(os.path.join(GEN, "splines.json")) as f:
        return json.load(f)["splines"]


def _poly(d):
    return [(tuple(int(e) for e in k.split(",")), Fraction(v)) for k, v in d.items()]


def _piece_of(tab, y):
    """Plane sign code of a folded offset and the piece sigma gives."""
    q = 0
    for i, (p, e) in enumerate(tab["planes"]):
        if sum(Fraction(pi) * yi for pi, yi in zip(p, y)) - Fraction(e) >= 0:
            q |= 1 << i
    return tab["sigma"][q % tab["r"]]


def table_eval(tab, coeffs, x):
    """f(x) from the generator's tables in exact rational arithmetic (x exact)."""
    s, D = tab["s"], tab["D"]
    dims = coeffs.shape[1:]
    total = Fraction(0)
    for k, l in enumerate(tab["cosets"]):
        u = [Fraction(x[a]) - l[a] for a in range(s)]
        i = [math.floor(u[a] / D + Fraction(1, 2)) for a in range(s)]
        y = [u[a] - D * i[a] for a in range(s)]
        order = sorted(range(s), key=lambda a: -abs(y[a]))       # folded slot -> original axis
        yf = [abs(y[a]) for a in order]
        sg = [(-1 if y[a] < 0 else 1) for a in order]
        pc = tab["pieces"][_piece_of(tab, yf)]
        t = [yf[a] - Fraction(pc["anchor"][a]) for a in range(s)]
        for g, P in zip(pc["sites"], pc["polys"]):
            idx = list(i)
            for a in range(s):
                idx[order[a]] += sg[a] * g[a]
            if all(0 <= idx[a] < dims[a] for a in range(s)):
                w = sum(v * math.prod(t[a] ** e[a] for a in range(s)) for e, v in _poly(P))
                total += Fraction(float(coeffs[(k,) + tuple(idx)])) * w
    return total


@pytest.mark.parametrize("name", NAMES)
def test_tables_match_the_oracle(tables, name):
    tab = tables[name]
    sp = SPLINES[name]
    lat = LATTICES[sp.lattice]
    s = tab["s"]
    rng = np.random.default_rng(7)
    N = 6
    c = rng.uniform(-1, 1, (len(lat.cosets),) + (N,) * s)
    npts = 40 if s == 4 or tab["degree"] > 6 or name == "bcc_voronoi2" else 80
    pts = (np.round(rng.uniform(0, lat.D * N, (npts, s)) * 2 ** 12) / 2 ** 12)
    ref = OracleSpline(name).eval_sum(lat.D, lat.cosets, c, pts)
    got = np.array([float(table_eval(tab, c, x)) for x in pts])
    assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("name", NAMES)
def test_pieces_tile_the_folded_region_and_sigma_names_them(tables, name):
    tab = tables[name]
    s, D = tab["s"], tab["D"]
    rng = np.random.default_rng(3)
    y = -np.sort(-rng.uniform(0, D / 2, (3000, s)), axis=1)          # uniform in the chamber
    polys = []
    for pc in tab["pieces"]:
        A = np.array([[float(Fraction(a)) for a in row[0]] for row in pc["ineqs"]])
        b = np.array([float(Fraction(row[1])) for row in pc["ineqs"]])
        polys.append((A, b))
    vols = np.zeros(len(polys))
    for yy in y:
        inside = [j for j, (A, b) in enumerate(polys) if np.all(A @ yy <= b + 1e-12)]
        assert len(inside) == 1
        assert _piece_of(tab, [Fraction(v) for v in yy]) == inside[0]
        vols[inside[0]] += 1
    frac = np.array([pc["volume_fraction"] for pc in tab["pieces"]])
    assert abs(frac.sum() - 1) < 1e-9
    assert np.abs(vols / len(y) - frac).max() < 0.04


@pytest.mark.parametrize("name", NAMES)
def test_mean_stencil_size_is_table1_lookups(tables, name):
    tab = tables[name]
    mean = len(tab["cosets"]) * sum(pc["volume_fraction"] * len(pc["sites"]) for pc in tab["pieces"])
    assert abs(mean - TABLE1_LOOKUPS[name]) < 1e-9
    assert abs(tab["lookups"] - TABLE1_LOOKUPS[name]) < 1e-9


def test_header_matches_a_fresh_generator_run(tables):
    from paper_2102_08514_b300.gen import analyse, CATALOG
    from paper_2102_08514_b300.gen.emit import HALF_STORAGE, emit_struct
    hdr = open(os.path.join(GEN, "splines.h")).read()
    for name in ("bcc_linear", "fcc_6dir"):
        L, xi = CATALOG[name]
        text, meta = emit_struct(analyse(name, L, xi), half_storage=name in HALF_STORAGE)
        assert text in hdr, name
        assert meta["sigma"] == tables[name]["sigma"]
    names = re.search(r"#define INTERP_GEN_SPLINES\(X\) (.*)", hdr).group(1)
    assert re.findall(r"X\((\w+)\)", names) == NAMES


def test_voronoi_expansion_sizes_are_the_papers():
    # Sec. 3: the BCC Voronoi region is 16 constant box splines, V_1 a sum of 136 box splines and
    # V_2 of 816 (before equal terms are merged); the FCC region (rhombic dodecahedron) is 4
    from math import comb
    from paper_2102_08514_b300.gen.catalog import G_BCC_VORONOI, G_FCC_VORONOI
    from paper_2102_08514_b300.gen.pieces import voronoi_terms, zonotope_tiling
    nb = len(zonotope_tiling([tuple(Fraction(v) for v in g) for g in G_BCC_VORONOI]))
    assert nb == 16 and comb(nb + 1, 2) == 136 and comb(nb + 2, 3) == 816
    assert len(zonotope_tiling([tuple(Fraction(v) for v in g) for g in G_FCC_VORONOI])) == 4
    for G, det_l in ((G_BCC_VORONOI, 4), (G_FCC_VORONOI, 2)):
        for order in (1, 2):
            terms = voronoi_terms(G, order, det_l)
            assert sum(t.w for t in terms) == det_l          # each M integrates to 1
            assert all(len(t.cols) == 3 * (order + 1) for t in terms)


def test_fold_requires_the_symmetry():
    from paper_2102_08514_b300.gen.pieces import signed_permutation_invariant
    for name in NAMES:
        assert signed_permutation_invariant([list(r) for r in SPLINES[name].xi])
    # one body diagonal only: not invariant under the signed permutations
    assert not signed_permutation_invariant([[1, 0, 0, 1], [0, 1, 0, 1], [0, 0, 1, 1]])


def test_unfolded_analysis_of_an_asymmetric_spline():
    # the generator also handles splines without the symmetry (no fold, whole cube, Sec. 4.2's
    # plane bits and sigma over all pieces), checked against the oracle on a few points
    from paper_2102_08514_b300.gen import analyse
    from paper_2102_08514_b300.gen.emit import emit_struct
    L = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    xi = [[1, 0, 0, 1], [0, 1, 0, 1], [0, 0, 1, 1]]
    T = analyse("diag4", L, xi)
    assert T.fold == 0
    _, meta = emit_struct(T)
    s, D = 3, 1
    rng = np.random.default_rng(5)
    c = rng.uniform(-1, 1, (1, 6, 6, 6))
    pts = np.round(rng.uniform(1, 5, (30, 3)) * 2 ** 10) / 2 ** 10
    ref = oracle.eval_sum(oracle.Spline(np.asarray(xi), 1), D, [[0, 0, 0]], c, pts)
    for q, x in enumerate(pts):
        total = Fraction(0)
        u = [Fraction(v) for v in x]
        i = [math.floor(u[a] + Fraction(1, 2)) for a in range(s)]
        y = [u[a] - i[a] for a in range(s)]
        pc = meta["pieces"][_piece_of(meta, y)]
        t = [y[a] - Fraction(pc["anchor"][a]) for a in range(s)]
        for g, P in zip(pc["sites"], pc["polys"]):
            idx = [i[a] + g[a] for a in range(s)]
            if all(0 <= idx[a] < 6 for a in range(s)):
                w = sum(v * math.prod(t[a] ** e[a] for a in range(s)) for e, v in _poly(P))
                total += Fraction(float(c[(0,) + tuple(idx)])) * w
        assert abs(float(total) - ref[q]) < 1e-12
