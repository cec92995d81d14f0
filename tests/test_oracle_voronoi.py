"""Pins of the oracle's Voronoi splines (Sec. 3: V_0 = chi, V_n = V_0 * V_{n-1}) to facts that do
not go through the oracle's own route (zonotope tiles, box-spline expansion):

* the tiles cover exactly the Voronoi region, defined as the points nearer to the origin than to
  any other lattice site;
* V_1(x) = vol(Vor n (x + Vor)) / |det L|^2 (the convolution of two indicators), computed from the
  region's half-spaces by scipy's half-space intersection and convex hull;
* partition of unity, reproduction of linear polynomials, and (V_2) the second-moment identity
  sum_n phi(x - n) n n^T = x x^T + (n+1) Cov(chi), with Cov(chi) integrated exactly over a
  tetrahedral decomposition of the Voronoi region;
* two different tilings (two choices of generic heights) give the same V_n;
* V_2(x) pointwise against its definition chi * chi * chi: the 6-D volume of
  {(y, w) : y, w, y + w - x in the Voronoi region}, from the region's half-spaces (qhull).
"""
import numpy as np
import pytest
from fractions import Fraction as Fr

import oracle
from synth import LATTICES, SPLINES

VORONOI = ["bcc_voronoi1", "bcc_voronoi2", "fcc_voronoi1", "fcc_voronoi2"]


def _spec(name):
    sp = SPLINES[name]
    lat = LATTICES[sp.lattice]
    gens = [tuple(Fr(int(v), 2) for v in col) for col in np.asarray(sp.xi).T]
    return lat, gens, sp.order


def _relevant_vectors(L):
    """Lattice vectors with |v|^2 <= 8 (a superset of the Voronoi-relevant ones for BCC and FCC in
    the integer frame) -- from the membership test, not from any coset structure."""
    v = oracle.lattice_sites(L, [-2.0] * 3, [2.0] * 3).astype(np.float64)
    n2 = (v * v).sum(axis=1)
    return v[(n2 > 0) & (n2 <= 8)]


def _voronoi_halfspaces(L, shift=np.zeros(3)):
    """{y : (y - shift) . v <= |v|^2 / 2} as scipy's [A | -b] rows (A y - b <= 0)."""
    V = _relevant_vectors(L)
    b = (V * V).sum(axis=1) / 2 + V @ shift
    return np.hstack([V, -b[:, None]])


def _intersection_volume(L, x):
    from scipy.spatial import ConvexHull, HalfspaceIntersection
    hs = np.vstack([_voronoi_halfspaces(L), _voronoi_halfspaces(L, x)])
    try:
        pts = HalfspaceIntersection(hs, x / 2).intersections
        return ConvexHull(pts).volume
    except Exception:
        return 0.0          # empty or degenerate intersection


def _voronoi_vertices(L):
    from scipy.spatial import HalfspaceIntersection
    return np.unique(np.round(HalfspaceIntersection(_voronoi_halfspaces(L), np.zeros(3)).intersections, 12), axis=0)


@pytest.mark.parametrize("lattice", ["bcc", "fcc"])
def test_tiles_cover_exactly_the_voronoi_region(lattice):
    name = f"{lattice}_voronoi1"
    lat, gens, _ = _spec(name)
    v = oracle.VoronoiSpline(lat.L, gens, 0)
    assert sum(t[2] for t in v.tiles) == abs(round(np.linalg.det(np.array(lat.L))))
    ctr = np.array([float(sum(g[a] for g in gens)) / 2 for a in range(3)])
    inv = [(np.linalg.inv(np.array([[float(gens[b][a]) for b in B] for a in range(3)])), np.array([float(z) for z in zb]))
           for B, zb, _ in v.tiles]
    V = _relevant_vectors(lat.L)
    rng = np.random.default_rng(11)
    x = rng.uniform(-1.6, 1.6, (4000, 3))
    checked = 0
    for p in x:
        margin = ((V * V).sum(axis=1) / 2 - V @ p).min()      # > 0 inside, < 0 outside
        if abs(margin) < 1e-6:
            continue
        lam = [Binv @ (p + ctr - zb) for Binv, zb in inv]
        if any(np.any(np.abs(l) < 1e-9) or np.any(np.abs(l - 1) < 1e-9) for l in lam):
            continue
        hits = sum(bool(np.all((l > 0) & (l < 1))) for l in lam)
        assert hits == (1 if margin > 0 else 0), (p, hits, margin)
        checked += 1
    assert checked > 3500


@pytest.mark.parametrize("lattice", ["bcc", "fcc"])
def test_v1_is_the_self_convolution_of_the_indicator(lattice):
    lat, gens, _ = _spec(f"{lattice}_voronoi1")
    v = oracle.VoronoiSpline(lat.L, gens, 1)
    det = abs(round(np.linalg.det(np.array(lat.L))))
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.5, 1.5, (60, 3))
    x[:3] = [[0, 0, 0], [0.5, 0.25, 0], [1, 1, 0.5]]
    got = v.phi(x)
    ref = np.array([_intersection_volume(lat.L, p) / det for p in x])
    assert np.abs(got - ref).max() < 1e-10
    assert (ref > 0).sum() > 20


def _second_moment(L):
    """Cov of the uniform distribution on the Voronoi region: exact per-tetrahedron moments."""
    from scipy.spatial import Delaunay
    P = _voronoi_vertices(L)
    tri = Delaunay(P)
    vol, S = 0.0, np.zeros((3, 3))
    for t in tri.simplices:
        v = P[t]
        tv = abs(np.linalg.det(v[1:] - v[0])) / 6
        ssum = v.sum(axis=0)
        S += tv / 20 * (v.T @ v + np.outer(ssum, ssum))
        vol += tv
    return vol, S / vol


@pytest.mark.parametrize("name", VORONOI)
def test_partition_of_unity_and_moments(name):
    lat, gens, order = _spec(name)
    v = oracle.VoronoiSpline(lat.L, gens, order)
    det = abs(round(np.linalg.det(np.array(lat.L))))
    vol, cov = _second_moment(lat.L)
    assert abs(vol - det) < 1e-12
    sites = oracle.lattice_sites(lat.L, [-7.0] * 3, [7.0] * 3).astype(np.float64)
    rng = np.random.default_rng(3)
    for x in rng.uniform(-1, 1, (4 if order > 1 else 8, 3)):
        w = v.phi(x - sites)
        assert abs(w.sum() - 1) < 1e-12
        assert np.abs(w @ sites - x).max() < 1e-11
        if order >= 2:
            # V_n's Fourier transform vanishes to order n + 1 at the nonzero dual lattice points
            # (chi's to order 1), so V_2 reproduces quadratics: the sum is the second moment
            m2 = (sites * w[:, None]).T @ sites
            assert np.abs(m2 - np.outer(x, x) - (order + 1) * cov).max() < 1e-10


@pytest.mark.parametrize("name", ["bcc_voronoi1", "fcc_voronoi2"])
def test_v_n_does_not_depend_on_the_tiling(name):
    lat, gens, order = _spec(name)
    a = oracle.VoronoiSpline(lat.L, gens, order)
    b = oracle.VoronoiSpline(lat.L, gens, order, heights=[Fr(-(j + 1) ** 2) for j in range(len(gens))])
    assert sorted(t[:2] for t in a.tiles) != sorted(t[:2] for t in b.tiles)      # another tiling
    x = np.random.default_rng(9).uniform(-2.5, 2.5, (40, 3))
    pa, ga = a.phi(x, grad=True)
    pb, gb = b.phi(x, grad=True)
    assert np.abs(pa - pb).max() < 1e-13
    assert np.abs(ga - gb).max() < 1e-12


def test_gradient_matches_finite_differences():
    lat, gens, order = _spec("bcc_voronoi2")
    v = oracle.VoronoiSpline(lat.L, gens, order)
    x = np.random.default_rng(2).uniform(-2, 2, (6, 3))
    _, g = v.phi(x, grad=True)
    h = 2.0 ** -20
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (v.phi(x + e) - v.phi(x - e)) / (2 * h)
        assert np.abs(fd - g[:, a]).max() < 1e-6


@pytest.mark.parametrize("name", ["bcc_voronoi1", "fcc_voronoi1", "cc_voronoi1", "bcc_linear"])
def test_gradient_at_exact_ties_is_the_one_sided_limit(name):
    # every decision, the gradient included, is the limit along x + eps v with the oracle's
    # v = (1, 2^-12, 2^-24) (direction); at points exactly on mesh planes and support boundaries
    # of a continuous, not C^1 spline the gradient must equal that limit
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from _gpu_common import OracleSpline
    sp = SPLINES[name]
    lat = LATTICES[sp.lattice]
    o = OracleSpline(name)
    c = np.random.default_rng(21).uniform(-1, 1, (len(lat.cosets), 9, 9, 9))
    rng = np.random.default_rng(22)
    x = np.round(rng.uniform(5, 12, (40, 3)) * 2) / 2              # integers and halves: ties
    x[::2, 2] += np.round(rng.uniform(0, 1, 20) * 2 ** 10) / 2 ** 10
    v = np.array([1.0, 2.0 ** -12, 2.0 ** -24])
    f0, g0 = o.eval_sum(lat.D, lat.cosets, c, x, grad=True)
    f1, g1 = o.eval_sum(lat.D, lat.cosets, c, x + 2.0 ** -36 * v, grad=True)
    assert np.abs(f0 - f1).max() < 1e-9
    assert np.abs(g0 - g1).max() < 1e-9


def test_table1_voronoi_rows(golden_dir):
    # Table 1's Voronoi rows on their own lattices: '# Lookups' (sites whose shifted basis is
    # nonzero at a generic point) and 'Order' (discrete moments constant below it, Strang-Fix)
    import itertools, json, os
    rows = json.load(open(os.path.join(golden_dir, "table1_lookups.json")))["voronoi_rows"]
    rng = np.random.default_rng(41)
    for row in rows:
        lat, gens, order = _spec(row["spline"])
        v = oracle.VoronoiSpline(lat.L, gens, order)
        assert order == row["order"] - 1                       # V_n has order n + 1
        xs = np.round(rng.uniform(-1, 1, (4, 3)) * 2 ** 18) / 2 ** 18
        betas = [b for d in range(row["order"] + 1) for b in itertools.product(range(d + 1), repeat=3) if sum(b) == d]
        moments = {}
        for x in xs:
            sites = oracle.lattice_sites(lat.L, x - v.halfwidth - 1, x + v.halfwidth + 1).astype(np.float64)
            w = v.phi(x - sites)
            assert int((w > 0).sum()) == row["lookups"], row["name"]
            for b in betas:
                moments.setdefault(b, []).append(np.sum(w * np.prod((sites - x) ** np.asarray(b), axis=1)))
        for b, m in moments.items():
            if sum(b) < row["order"]:
                assert np.ptp(m) < 1e-9, (row["name"], b)
        assert max(np.ptp(m) for b, m in moments.items() if sum(b) == row["order"]) > 1e-6, row["name"]


def _vol6_triple_overlap(L, x):
    """6-D volume of {(y, w) : y, w and y + w - x all in the Voronoi region}: with chi the indicator
    of the region scaled by 1/|det L|, V_2 = chi * chi * chi gives
    phi(x) = |det L| V_2(x) = vol / |det L|^2.  Half-spaces from the membership-derived relevant
    vectors; interior point by linear programming (Chebyshev centre); volume by qhull in 6-D."""
    from scipy.optimize import linprog
    from scipy.spatial import ConvexHull, HalfspaceIntersection
    V = _relevant_vectors(L)
    b = (V * V).sum(axis=1) / 2
    n = len(V)
    A = np.zeros((3 * n, 6))
    rhs = np.zeros(3 * n)
    A[:n, :3], rhs[:n] = V, b
    A[n:2 * n, 3:], rhs[n:2 * n] = V, b
    A[2 * n:, :3], A[2 * n:, 3:], rhs[2 * n:] = V, V, b + V @ x
    norms = np.linalg.norm(A, axis=1)
    lp = linprog(np.r_[np.zeros(6), -1.0], A_ub=np.c_[A, norms], b_ub=rhs, bounds=[(None, None)] * 6 + [(0, None)])
    if lp.status != 0 or lp.x[-1] < 1e-9:
        return 0.0
    pts = HalfspaceIntersection(np.c_[A, -rhs], lp.x[:6]).intersections
    # the polytope is not simple (more than 6 facets meet at some vertices): qhull with its exact
    # pre-merge and wide merges allowed; it agrees to rounding at most points, to ~1e-7 at a few
    return ConvexHull(pts, qhull_options="Qx Q12").volume


@pytest.mark.parametrize("lattice,npts", [("bcc", 5), ("fcc", 8)])
def test_v2_is_the_triple_convolution_of_the_indicator(lattice, npts):
    # pointwise pin of V_2 against its definition, independent of the oracle's tiling and
    # box-spline expansion: phi(x) = vol{(y, w) : y, w, y + w - x in Vor} / |det L|^2
    lat, gens, _ = _spec(f"{lattice}_voronoi2")
    v = oracle.VoronoiSpline(lat.L, gens, 2)
    det = abs(round(np.linalg.det(np.array(lat.L))))
    rng = np.random.default_rng(17)
    x = rng.uniform(-1.6, 1.6, (npts, 3))
    x[0] = (0.0123, 0.0456, 0.0789)     # near the centre, off its symmetry planes (generic for qhull)
    got = v.phi(x)
    ref = np.array([_vol6_triple_overlap(lat.L, p) / det ** 2 for p in x])
    assert np.all(ref > 0)
    rel = np.abs(got - ref) / ref
    # a dropped term or a wrong weight shows at 1e-3 or more; qhull's wide merges stay below 1e-6
    assert rel.max() < 1e-6, rel
    assert np.median(rel) < 1e-12, rel
