"""Pins of the CPU oracle to facts the paper and the mathematics fix (no GPU).

Each test ties the oracle to something other than itself: textbook closed forms (cardinal
B-splines, the bilinear hat of Xi_TP2, the quincunx example Xi_QC of Sec. 4), the values the paper
prints (Table 1 '# Lookups' and 'Order', Sec. 5.2's 240/60 accesses), and invariants (integral 1,
partition of unity on L, support = zonotope, signed-permutation symmetry, Strang-Fix moments,
C^(m-2) continuity, the closed-form directional derivative against finite differences, the
adjoint dot-product identity, the coset decomposition of Sec. 4.1 against a direct lattice sum).
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import Spline, lattice_sites
from synth import LATTICES, SPLINES

RNG = np.random.default_rng(20210217)


def dyadic(x, bits=20):
    """Round to a multiple of 2^-bits so that every shifted copy is exact in FP64."""
    return np.round(np.asarray(x) * 2.0 ** bits) / 2.0 ** bits


def spline_of(name):
    sp = SPLINES[name]
    lat = LATTICES[sp.lattice]
    detl = abs(round(np.linalg.det(np.asarray(lat.L, dtype=float))))
    return Spline(np.asarray(sp.xi), detl), lat


def zonotope_h(xi):
    """H-representation of the centred zonotope: normals of (s-1)-subsets, half-widths."""
    xi = np.asarray(xi)
    s, n = xi.shape
    out = {}
    for sub in itertools.combinations(range(n), s - 1):
        V = xi[:, sub].T.astype(float)
        if s == 1:
            p = np.array([1.0])
        else:
            p = np.array([(-1) ** i * np.linalg.det(np.delete(V, i, axis=1)) for i in range(s)])
        if np.abs(p).max() < 0.5:
            continue
        p = p / np.abs(p).max()
        key = tuple(np.round(p * 1e6).astype(int))
        out[key] = (p, 0.5 * np.abs(p @ xi).sum())
    return list(out.values())


# ----------------------------------------------------------------------------- closed forms

def cardinal_bspline(n, x):
    """M_n(x) = 1/(n-1)! sum_k (-1)^k C(n,k) (x-k)_+^(n-1), the textbook truncated-power form."""
    if n == 1:
        return 1.0 if 0 <= x < 1 else 0.0
    tot = 0.0
    for k in range(n + 1):
        t = x - k
        if t > 0:
            tot += (-1) ** k * math.comb(n, k) * t ** (n - 1)
    return tot / math.factorial(n - 1)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_1d_cardinal_bspline(n):
    sp = Spline([[1] * n])
    xs = dyadic(RNG.uniform(-0.5, n + 0.5, 64))
    got = sp.M(xs[:, None])
    ref = np.array([cardinal_bspline(n, x) for x in xs])
    assert np.abs(got - ref).max() < 1e-12


def test_2d_tp2_is_bilinear_hat():
    # Sec. 4 running example Xi_TP2 = [[1,0,-1,0],[0,1,0,-1]]: centred, it is the bilinear hat
    sp = Spline([[1, 0, -1, 0], [0, 1, 0, -1]], det_l=1)
    z = dyadic(RNG.uniform(-1.3, 1.3, (200, 2)))
    ref = np.clip(1 - np.abs(z[:, 0]), 0, None) * np.clip(1 - np.abs(z[:, 1]), 0, None)
    assert np.abs(sp.phi(z) - ref).max() < 1e-13


def test_2d_quincunx_example():
    # Sec. 4: Xi_QC = [[2,0,-2,0],[0,2,0,-2]] on L_QC = [[1,-1],[1,1]] (|det| = 2).  M_{2 Xi} =
    # M_Xi(x/2)/4, so phi = 2 M_QC = (1 - |x|/2)_+ (1 - |y|/2)_+ / 2; partition of unity on L_QC.
    LQC = [[1, -1], [1, 1]]
    sp = Spline([[2, 0, -2, 0], [0, 2, 0, -2]], det_l=2)
    z = dyadic(RNG.uniform(-2.5, 2.5, (200, 2)))
    ref = 0.5 * np.clip(1 - np.abs(z[:, 0]) / 2, 0, None) * np.clip(1 - np.abs(z[:, 1]) / 2, 0, None)
    assert np.abs(sp.phi(z) - ref).max() < 1e-13
    for x in dyadic(RNG.uniform(-3, 3, (10, 2))):
        sites = lattice_sites(LQC, x - 3, x + 3)
        assert abs(sp.phi(x - sites).sum() - 1.0) < 1e-13


def test_3d_tensor_products():
    I = np.eye(3, dtype=int)
    z = dyadic(RNG.uniform(-1.8, 1.8, (100, 3)))
    lin = Spline(np.hstack([I, I]))
    ref = np.prod(np.clip(1 - np.abs(z), 0, None), axis=1)
    assert np.abs(lin.phi(z) - ref).max() < 1e-13

    def b2(t):
        t = np.abs(t)
        return np.where(t <= 0.5, 0.75 - t * t, np.where(t <= 1.5, 0.5 * (1.5 - t) ** 2, 0.0))

    quad = Spline(np.hstack([I, I, I]))
    assert np.abs(quad.phi(z) - np.prod(b2(z), axis=1)).max() < 1e-13


# ----------------------------------------------------------------------------- invariants

CONFIG_SPLINES = ["bcc_linear", "bcc_quintic", "fcc_6dir", "cc_7dir", "d4s_8dir"]


@pytest.mark.parametrize("name", ["bcc_linear", "fcc_6dir", "cc_7dir", "bcc_quintic"])
def test_integral_is_one(name):
    # Riemann sum on the grid h Z^s with h = 1/2: M_Xi(h.) = h^-s M_{Xi/h}, and Xi/h is integer,
    # whose integer translates sum to 1, so the sum h^s sum_k M_Xi(h k + o) equals the integral 1
    # exactly for every offset o.
    sp = SPLINES[name]
    xi = np.asarray(sp.xi)
    s = xi.shape[0]
    M = Spline(xi)
    lo = np.minimum(xi, 0).sum(axis=1)
    hi = np.maximum(xi, 0).sum(axis=1)
    h = 0.5
    for o in dyadic(RNG.uniform(0, h, (2, s)), 12):
        axes = [np.arange(np.floor((lo[a] - o[a]) / h), np.ceil((hi[a] - o[a]) / h) + 1) * h + o[a]
                for a in range(s)]
        grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, s)
        assert abs(M.M(grid).sum() * h ** s - 1.0) < 1e-12


@pytest.mark.parametrize("name", CONFIG_SPLINES)
def test_partition_of_unity_and_linear_reproduction(name):
    sp, lat = spline_of(name)
    h = sp.halfwidth
    for x in dyadic(RNG.uniform(-3, 3, (6, sp.s))):
        sites = lattice_sites(lat.L, x - h - 1, x + h + 1)
        w = sp.phi(x - sites)
        assert abs(w.sum() - 1.0) < 1e-12
        assert np.abs(w @ sites - x).max() < 1e-11


@pytest.mark.parametrize("name", CONFIG_SPLINES)
def test_cosets_generate_lattice(name):
    # D Z^s + {l_k} (the coset split of Sec. 4.1) is exactly L Z^s
    _, lat = spline_of(name)
    s = len(lat.L)
    box = lattice_sites(lat.L, [0] * s, [2 * lat.D - 1] * s)
    from_cosets = {tuple(np.asarray(l) + lat.D * np.asarray(g))
                   for l in lat.cosets for g in itertools.product(range(2), repeat=s)}
    assert {tuple(v) for v in box} == from_cosets


def test_table1_lookups_and_order(golden_dir):
    rows = json.load(open(os.path.join(golden_dir, "table1_lookups.json")))["rows"]
    for row in rows:
        xi = np.asarray(row["xi"])
        L = np.asarray(row["L"])
        detl = abs(round(np.linalg.det(L)))
        sp = Spline(xi, detl)
        s = xi.shape[0]
        h = sp.halfwidth
        nx = 3 if s == 4 else 5
        xs = dyadic(RNG.uniform(-1, 1, (nx, s)), 18)
        moments = {}
        order = row["order"]
        betas = [b for d in range(order + 1) for b in itertools.product(range(d + 1), repeat=s) if sum(b) == d]
        for x in xs:
            sites = lattice_sites(L, x - h - 1, x + h + 1)
            w = sp.phi(x - sites)
            # '# Lookups': sites whose shifted basis is nonzero at a generic point
            assert int((w > 0).sum()) == row["lookups"], row["name"]
            for b in betas:
                moments.setdefault(b, []).append(np.sum(w * np.prod((sites - x) ** np.asarray(b), axis=1)))
        # 'Order' m (Strang-Fix): discrete moments sum_n (n-x)^b phi(x-n) are constant in x for
        # |b| < m, and some moment of degree m is not
        for b, v in moments.items():
            spread = np.ptp(v)
            if sum(b) < order:
                assert spread < 1e-9, (row["name"], b, spread)
        assert max(np.ptp(v) for b, v in moments.items() if sum(b) == order) > 1e-4, row["name"]


@pytest.mark.parametrize("name", CONFIG_SPLINES)
def test_support_is_the_zonotope(name):
    sp, _ = spline_of(name)
    H = zonotope_h(np.asarray(SPLINES[name].xi))
    z = dyadic(RNG.uniform(-1, 1, (1500, sp.s)) * (0.8 * sp.halfwidth + 0.3))
    slack = np.min([hw - np.abs(z @ p) for p, hw in H], axis=0)
    v = sp.phi(z)
    assert np.all(v[slack < -1e-9] == 0.0)
    assert np.all(v[slack > 1e-9] > 0.0)
    assert (slack > 1e-9).sum() > 50 and (slack < -1e-9).sum() > 50


@pytest.mark.parametrize("name", CONFIG_SPLINES)
def test_signed_permutation_symmetry(name):
    sp, _ = spline_of(name)
    s = sp.s
    z = dyadic(RNG.uniform(-1, 1, (4, s)) * sp.halfwidth)
    base = sp.phi(z)
    for perm in itertools.permutations(range(s)):
        for signs in itertools.product((1, -1), repeat=s):
            zz = z[:, perm] * np.asarray(signs)
            assert np.abs(sp.phi(zz) - base).max() < 1e-12


@pytest.mark.parametrize("name", CONFIG_SPLINES)
def test_two_solutions_of_xi_t_agree(name):
    # the recurrence is valid for any t with Xi t = x; two different choices must agree
    sp = SPLINES[name]
    a = Spline(np.asarray(sp.xi), tmode=0)
    b = Spline(np.asarray(sp.xi), tmode=1)
    w = dyadic(RNG.uniform(-0.2, 1.2, (300, a.s)) * np.maximum(np.asarray(sp.xi), 0).sum(axis=1))
    assert np.abs(a.M(w) - b.M(w)).max() < 1e-12


@pytest.mark.parametrize("name", CONFIG_SPLINES)
def test_gradient_closed_form_vs_central_differences(name):
    sp, _ = spline_of(name)
    s = sp.s
    z = dyadic(RNG.uniform(-1, 1, (40, s)) * sp.halfwidth * 0.8)
    v, g = sp.phi(z, grad=True)
    h = 2.0 ** -18
    for a in range(s):
        e = np.zeros(s)
        e[a] = h
        fd = (sp.phi(z + e) - sp.phi(z - e)) / (2 * h)
        assert np.abs(fd - g[:, a]).max() < 1e-6


def _points_on_mesh_planes(xi, count):
    """Dyadic points exactly on mesh planes p . x = d of the centred spline (Sec. 3, the mesh)."""
    xi = np.asarray(xi)
    s, n = xi.shape
    c = xi.sum(axis=1) / 2.0
    out = []
    while len(out) < count:
        sub = RNG.choice(n, s - 1, replace=False)
        V = xi[:, sub].T.astype(float)
        p = np.round([(-1) ** i * np.linalg.det(np.delete(V, i, axis=1)) for i in range(s)]).astype(int)
        if not p.any():
            continue
        p = p // np.gcd.reduce(np.abs(p[p != 0]))
        A = RNG.random(n) < 0.5
        d = p @ (xi[:, A].sum(axis=1) - c)
        k = int(np.argmax(np.abs(p)))
        x = dyadic(RNG.uniform(-1, 1, s) * 1.5, 10)
        x[k] = 0.0
        x[k] = (d - p @ x) / p[k]
        out.append((x, p / np.linalg.norm(p)))
    return out


@pytest.mark.parametrize("name,order", [("bcc_linear", 2), ("bcc_quintic", 4), ("fcc_6dir", 3),
                                        ("cc_7dir", 4)])
def test_smoothness_across_mesh_planes(name, order):
    # box splines are C^(m-2) (Sec. 3 / de Boor): values are continuous across every mesh plane;
    # the gradient is continuous too when m >= 3 and jumps somewhere when m = 2
    sp, _ = spline_of(name)
    h = 2.0 ** -24
    max_gjump = 0.0
    for x, nrm in _points_on_mesh_planes(SPLINES[name].xi, 60):
        zp = x + h * nrm
        zm = x - h * nrm
        (vp,), gp = sp.phi(zp[None], grad=True)
        (vm,), gm = sp.phi(zm[None], grad=True)
        assert abs(vp - vm) < 1e-5
        max_gjump = max(max_gjump, np.abs(gp - gm).max())
    if order >= 3:
        assert max_gjump < 1e-4
    else:
        assert max_gjump > 1e-2


@pytest.mark.parametrize("name", CONFIG_SPLINES)
def test_coset_sum_equals_direct_lattice_sum(name):
    # the coset form of Sec. 4.1 against a direct sum over L Z^s (membership enumeration)
    sp, lat = spline_of(name)
    s = sp.s
    N = 6
    shape = (len(lat.cosets),) + (N,) * s
    c = RNG.uniform(-1, 1, shape)
    lookup = {}
    for k, l in enumerate(lat.cosets):
        for i in itertools.product(range(N), repeat=s):
            lookup[tuple(lat.D * np.asarray(i) + np.asarray(l))] = c[(k,) + i]
    pts = dyadic(RNG.uniform(0, lat.D * N, (20, s)))
    got = oracle.eval_sum(sp, lat.D, lat.cosets, c, pts)
    h = sp.halfwidth
    for q, x in enumerate(pts):
        sites = lattice_sites(lat.L, x - h - 1, x + h + 1)
        w = sp.phi(x - sites)
        ref = sum(wi * lookup.get(tuple(n), 0.0) for wi, n in zip(w, sites))
        assert abs(got[q] - ref) < 1e-12


@pytest.mark.parametrize("name", ["bcc_linear", "fcc_6dir", "d4s_8dir"])
def test_adjoint_dot_product_and_gradient(name):
    sp, lat = spline_of(name)
    s = sp.s
    N = 5
    shape = (len(lat.cosets),) + (N,) * s
    c = RNG.uniform(-1, 1, shape)
    pts = dyadic(RNG.uniform(0, lat.D * N, (30, s)))
    g = RNG.uniform(-1, 1, 30)
    f, grad = oracle.eval_sum(sp, lat.D, lat.cosets, c, pts, grad=True)
    dc = oracle.adjoint(sp, lat.D, lat.cosets, shape, pts, g)
    assert abs(f @ g - np.sum(c * dc)) < 1e-11
    hh = 2.0 ** -18
    for a in range(s):
        e = np.zeros(s)
        e[a] = hh
        fd = (oracle.eval_sum(sp, lat.D, lat.cosets, c, pts + e) - oracle.eval_sum(sp, lat.D, lat.cosets, c, pts - e)) / (2 * hh)
        assert np.abs(fd - grad[:, a]).max() < 1e-6


def test_cells_are_the_exact_rounding():
    lat = LATTICES["bcc"]
    pts = RNG.uniform(-5, 40, (200, 3)).astype(np.float32).astype(np.float64)
    pts[:10] = np.round(pts[:10])            # exact ties on cell boundaries
    ci, off = oracle.cells(3, lat.D, lat.cosets, pts)
    for q in range(len(pts)):
        for k, l in enumerate(lat.cosets):
            for a in range(3):
                u = Fraction(pts[q, a]) - l[a]
                i = math.floor(u / lat.D + Fraction(1, 2))
                assert ci[q, k, a] == i
                y = u - lat.D * i
                assert Fraction(off[q, k, a]) == y and -1 <= y < 1


def test_folded_offsets_land_in_the_chamber():
    y = RNG.uniform(-1, 1, (500, 4))
    f = oracle.folded_offsets(y)
    assert np.all(f[:, :-1] >= f[:, 1:]) and np.all(f >= 0) and np.all(f <= 1)
    # a signed permutation of the input: same multiset of absolute values
    assert np.allclose(np.sort(np.abs(y), axis=1), np.sort(f, axis=1))
