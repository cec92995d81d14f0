"""Exact piecewise-polynomial analysis of phi(x) = |det L| M_Xi(x + sum(Xi)/2) per Cartesian coset.

Steps (Horacsek & Alim, arXiv 2102.08514):

1. Cartesian coset decomposition L Z^s = U_k (D Z^s + l_k) with G L = D = d I (Sec. 4.1).
2. Region of evaluation: the cube [-D/2, D/2)^s centred on the nearest coset site, so the shift
   rho(x) is a rounding (Sec. 4.1, the function rho).
3. Symmetry fold: when every signed permutation S maps Xi onto itself up to column signs, phi is
   invariant under S, and the cube folds onto the chamber D/2 >= y_1 >= ... >= y_s >= 0.  This is
   the reflection trick of Sec. 4.2 taken to the whole signed-permutation group; the per-piece
   change of variables (T, t, pi) of Sec. 4.3 becomes the per-query signed permutation S.
4. Sub-regions: the mesh planes of Sec. 3 (hyperplanes spanned by (s-1)-subsets of Xi, through
   every sum of a subset of the columns, shifted by D Z^s) that cut the chamber; their cells are the
   sub-regions of evaluation S_j (Sec. 4.1), identified branch-free by plane sign bits q and a
   table sigma[q] (Sec. 4.2; uncompressed, so that codes of points on planes map to an adjacent
   piece -- see _sigma_table).
5. Per cell, the stencil C_0(S_j) (the coset sites whose shifted support covers the cell) and the
   explicit polynomial of phi(y - D g) for every stencil site g (the functions psi_j of Sec. 4.1).
   The polynomials are computed exactly (Fractions) by running de Boor's recurrence on polynomials
   in y: inside one cell every sub-box-spline M_{Xi'}(y + v) is a single polynomial, and every
   base-case decision is constant on the cell, so it is taken at an interior point.

Everything here is exact rational arithmetic; the emitter rounds to FP32 only at the end.
"""
from __future__ import annotations

import itertools
import math
import os
from dataclasses import dataclass, field
from fractions import Fraction as Fr
from functools import lru_cache


# ----------------------------------------------------------------------------- exact linear algebra

def det(m):
    """Determinant of a small square matrix of ints/Fractions (Laplace expansion)."""
    n = len(m)
    if n == 1:
        return m[0][0]
    if n == 2:
        return m[0][0] * m[1][1] - m[0][1] * m[1][0]
    total = 0
    for c in range(n):
        if m[0][c] == 0:
            continue
        sub = [row[:c] + row[c + 1:] for row in m[1:]]
        total += (-1) ** c * m[0][c] * det(sub)
    return total


def solve(A, b):
    """Exact solution of A x = b (A square, nonsingular) by Gauss-Jordan over Fractions."""
    n = len(A)
    M = [[Fr(v) for v in A[r]] + [Fr(b[r])] for r in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        pv = M[c][c]
        M[c] = [v / pv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * bb for a, bb in zip(M[r], M[c])]
    return [M[r][n] for r in range(n)]


def inverse(A):
    n = len(A)
    cols = [solve(A, [1 if i == j else 0 for i in range(n)]) for j in range(n)]
    return [[cols[j][i] for j in range(n)] for i in range(n)]


def rank(vectors, s):
    rows = [[Fr(v) for v in vec] for vec in vectors]
    r = 0
    for c in range(s):
        p = next((i for i in range(r, len(rows)) if rows[i][c] != 0), None)
        if p is None:
            continue
        rows[r], rows[p] = rows[p], rows[r]
        for i in range(len(rows)):
            if i != r and rows[i][c] != 0:
                f = rows[i][c] / rows[r][c]
                rows[i] = [a - f * b for a, b in zip(rows[i], rows[r])]
        r += 1
    return r


def hyperplane_normal(vectors, s):
    """Primitive integer normal of the hyperplane spanned by s-1 integer vectors (None if they do
    not span a hyperplane); sign fixed so that the first nonzero entry is positive."""
    n = []
    for i in range(s):
        sub = [[Fr(v[k]) for k in range(s) if k != i] for v in vectors]
        n.append((-1) ** i * det(sub) if s > 1 else Fr(1))
    den = 1
    for a in n:
        den = den * Fr(a).denominator // math.gcd(den, Fr(a).denominator)
    n = [Fr(a) * den for a in n]
    g = 0
    for a in n:
        g = math.gcd(g, abs(int(a)))
    if g == 0:
        return None
    n = [int(a) // g for a in n]
    for a in n:
        if a != 0:
            if a < 0:
                n = [-b for b in n]
            break
    return tuple(n)


# ----------------------------------------------------------------------------- lattice structure

def coset_structure(L):
    """D (with D Z^s inside L Z^s, D minimal) and the coset shifts l_k in [0, D)^s (Sec. 4.1)."""
    s = len(L)
    dl = det(L)
    if dl == 0:
        raise ValueError("L must have full rank")
    Linv = inverse(L)

    def member(z):
        return all(sum(Linv[i][j] * z[j] for j in range(s)).denominator == 1 for i in range(s))

    D = next(d for d in range(1, abs(dl) + 1)
             if all(member([d if j == i else 0 for j in range(s)]) for i in range(s)))
    cosets = [z for z in itertools.product(range(D), repeat=s) if member(z)]
    assert len(cosets) * abs(dl) == D ** s, "coset count must be D^s / |det L|"
    return D, [list(z) for z in cosets], abs(dl)


def signed_permutation_invariant(xi):
    """True if every signed permutation maps the columns of Xi onto themselves up to sign, i.e.
    the centred box spline is invariant under the whole hyperoctahedral group."""
    s = len(xi)
    cols = [tuple(xi[a][j] for a in range(s)) for j in range(len(xi[0]))]

    def canon(v):
        for a in v:
            if a != 0:
                return tuple(v) if a > 0 else tuple(-b for b in v)
        return tuple(v)

    base = sorted(canon(c) for c in cols)
    for perm in itertools.permutations(range(s)):
        for signs in itertools.product((1, -1), repeat=s):
            img = sorted(canon([signs[a] * c[perm[a]] for a in range(s)]) for c in cols)
            if img != base:
                return False
    return True


# ----------------------------------------------------------------------------- polynomials

def n_monomials(s, d):
    return math.comb(d + s, s)


@lru_cache(maxsize=None)
def horner_order(s, d):
    """Monomial exponent tuples of total degree <= d in s variables, in the nested-Horner layout
    the kernels use: P(t_1..t_s) = sum_k t_1^k P_k(t_2..t_s), with deg P_k <= d - k, stored as
    P_0, P_1, ..., P_d, each recursively in the same layout."""
    if s == 0:
        return ((),)
    out = []
    for k in range(d + 1):
        for rest in horner_order(s - 1, d - k):
            out.append((k,) + rest)
    return tuple(out)


class Poly:
    """Sparse polynomial with exact Fraction coefficients: {exponent tuple: Fraction}."""
    __slots__ = ("c",)

    def __init__(self, c=None):
        self.c = c or {}

    @staticmethod
    def const(v, s):
        return Poly({(0,) * s: Fr(v)}) if v != 0 else Poly()

    def is_zero(self):
        return not self.c

    def add(self, other, scale=1):
        out = dict(self.c)
        for e, v in other.c.items():
            w = out.get(e, 0) + scale * v
            if w:
                out[e] = w
            else:
                out.pop(e, None)
        return Poly(out)

    def scale(self, a):
        if a == 0:
            return Poly()
        return Poly({e: v * a for e, v in self.c.items()})

    def mul_affine(self, aff):
        """Multiply by a0 + sum_a aff[1+a] y_a."""
        s = len(aff) - 1
        out = {}
        for e, v in self.c.items():
            if aff[0]:
                w = out.get(e, 0) + v * aff[0]
                out[e] = w
            for a in range(s):
                if aff[1 + a]:
                    e2 = e[:a] + (e[a] + 1,) + e[a + 1:]
                    out[e2] = out.get(e2, 0) + v * aff[1 + a]
        return Poly({e: v for e, v in out.items() if v})

    def taylor_shift(self, anchor):
        """Return Q with Q(t) = P(t + anchor) (re-expansion about the anchor point)."""
        s = len(anchor)
        out = {}
        for e, v in self.c.items():
            # prod_a (t_a + anchor_a)^{e_a}
            terms = [{(): v}]
            for a in range(s):
                nxt = {}
                for pre, pv in terms[-1].items():
                    for k in range(e[a] + 1):
                        coef = pv * math.comb(e[a], k) * (anchor[a] ** (e[a] - k))
                        if coef:
                            key = pre + (k,)
                            nxt[key] = nxt.get(key, 0) + coef
                terms.append(nxt)
            for key, cv in terms[-1].items():
                out[key] = out.get(key, 0) + cv
        return Poly({e: v for e, v in out.items() if v})

    def __call__(self, y):
        tot = Fr(0)
        for e, v in self.c.items():
            term = v
            for a, k in enumerate(e):
                if k:
                    term *= Fr(y[a]) ** k
            tot += term
        return tot


# ----------------------------------------------------------------------------- polytopes

@dataclass
class Cell:
    """A convex polytope {y : a . y <= b for (a, b) in ineqs} with its exact vertices."""
    ineqs: list
    verts: list = field(default_factory=list)
    signs: dict = field(default_factory=dict)   # plane index -> 0/1 side bit

    def interior_point(self):
        n = len(self.verts)
        s = len(self.verts[0])
        return [sum(v[a] for v in self.verts) / n for a in range(s)]


def vertices(ineqs, s):
    """Vertices of {a . y <= b} by brute force over s-subsets of the inequalities."""
    vs = set()
    for sub in itertools.combinations(range(len(ineqs)), s):
        A = [ineqs[i][0] for i in sub]
        if det(A) == 0:
            continue
        y = solve(A, [ineqs[i][1] for i in sub])
        if all(sum(a[k] * y[k] for k in range(s)) <= b for a, b in ineqs):
            vs.add(tuple(y))
    return [list(v) for v in sorted(vs)]


def split(cell, p, e, s, idx):
    """Split a cell by the plane p . y = e if the plane passes through its interior."""
    vals = [sum(p[k] * v[k] for k in range(s)) - e for v in cell.verts]
    if not (any(v > 0 for v in vals) and any(v < 0 for v in vals)):
        side = 1 if any(v > 0 for v in vals) else 0
        cell.signs[idx] = side
        return [cell]
    out = []
    for side, (a, b) in ((0, (list(p), e)), (1, ([-x for x in p], -e))):
        ineqs = cell.ineqs + [(a, b)]
        c = Cell(ineqs, vertices(ineqs, s), dict(cell.signs))
        c.signs[idx] = side
        out.append(c)
    return out


# ----------------------------------------------------------------------------- the analysis

@dataclass
class Piece:
    anchor: list          # expansion point (exact rationals) of the piece polynomials
    sites: list           # grid offsets g (ints): coset site D*g relative to the nearest site
    polys: list           # exact Poly per site, in t = y - anchor
    code: int             # plane sign bits q of the cell
    verts: list           # exact vertices of the cell
    ineqs: list           # exact H-representation of the cell


@dataclass
class SplineTables:
    name: str
    s: int
    L: list
    xi: list
    det_l: int
    D: int
    cosets: list
    fold: int             # 2: signed permutations, 0: none
    degree: int
    planes: list          # (p: tuple of ints, e: Fraction) in the folded frame
    r: int                # sigma's length, 2^Q (the table is indexed by q directly)
    sigma: list           # sigma[q] -> piece index
    pieces: list
    halo: int             # max |g_a| over all stencil sites (grid units)
    lookups: int = 0      # coefficient reads per query (all cosets)
    kind: int = 0         # 0: box spline M_Xi; n >= 1: Voronoi spline V_n (xi records 2 G)
    smooth: int = 0       # phi is in C^smooth


@dataclass(frozen=True)
class Term:
    """One summand w * M_cols(x + c) of phi (cols: direction vectors as tuples of Fractions)."""
    w: Fr
    cols: tuple
    c: tuple


def box_spline_terms(xi, det_l):
    """phi = |det L| M_Xi(x + sum(Xi)/2), the centred box spline scaled to a partition of unity."""
    s, n = len(xi), len(xi[0])
    cols = tuple(tuple(Fr(xi[a][j]) for a in range(s)) for j in range(n))
    return [Term(Fr(det_l), cols, tuple(sum(c[a] for c in cols) / 2 for a in range(s)))]


def zonotope_tiling(gens):
    """Tiles of the zonotope Z(G) = sum_j [0, g_j] by parallelepipeds: a list of (B, z_B, |det B|)
    over the bases B of G with Z(G) = union of z_B + B[0,1)^s (disjoint up to boundaries).

    The tiles are the lower facets of the zonotope of the lifted generators (g_j, h_j) for generic
    heights h_j, projected back: the facet spanned by B has the normal (-a, 1) with a . g_b = h_b
    on B, and its offset is the sum of the g_j (j not in B) with h_j < a . g_j."""
    s, m = len(gens[0]), len(gens)
    for k in itertools.count(2):
        hts = [Fr((j + 1) ** k) for j in range(m)]
        tiles = []
        generic = True
        for B in itertools.combinations(range(m), s):
            GB = [[Fr(gens[b][a]) for b in B] for a in range(s)]
            dB = det(GB)
            if dB == 0:
                continue
            a_ = solve([[Fr(gens[b][a]) for a in range(s)] for b in B], [hts[b] for b in B])
            z = [Fr(0)] * s
            for j in range(m):
                if j in B:
                    continue
                d = hts[j] - sum(a_[a] * gens[j][a] for a in range(s))
                if d == 0:
                    generic = False
                    break
                if d < 0:
                    z = [z[a] + gens[j][a] for a in range(s)]
            if not generic:
                break
            tiles.append((B, tuple(z), abs(dB)))
        if generic:
            return tiles


def voronoi_terms(gens, order, det_l):
    """phi = |det L| V_order with V_0 = chi (1/|det L| on the Voronoi region), V_n = V_0 * V_{n-1}
    (Sec. 3), for a Voronoi region that is the centred zonotope of the generators G.

    V_0 = 1/|det L| sum_B |det B| M_B(x + sum(G)/2 - z_B) over the tiles (B, z_B) of Z(G); the
    (order+1)-fold convolution expands by the multinomial theorem into box splines of the
    concatenated bases (Sec. 3: convolving box splines concatenates their direction matrices and
    adds their shifts).  Equal (directions, shift) pairs are merged."""
    s = len(gens[0])
    gens = [tuple(Fr(v) for v in g) for g in gens]
    tiles = zonotope_tiling(gens)
    half = [sum(g[a] for g in gens) / 2 for a in range(s)]
    acc = {}
    for combo in itertools.combinations_with_replacement(range(len(tiles)), order + 1):
        mult = math.factorial(order + 1)
        for i in set(combo):
            mult //= math.factorial(combo.count(i))
        w = Fr(mult) * Fr(det_l) / Fr(det_l) ** (order + 1)
        for i in combo:
            w *= tiles[i][2]
        cols = tuple(sorted(gens[b] for i in combo for b in tiles[i][0]))
        c = tuple(sum(half[a] - tiles[i][1][a] for i in combo) for a in range(s))
        acc[(cols, c)] = acc.get((cols, c), 0) + w
    return [Term(w, cols, c) for (cols, c), w in sorted(acc.items())]


def _canon_dir(v):
    for a in v:
        if a != 0:
            return tuple(v) if a > 0 else tuple(-b for b in v)
    return tuple(v)


def analyse(name, L, xi, anchor_den=64, verbose=False):
    """Run the analysis for phi = |det L| M_Xi(. + sum(Xi)/2) on the lattice L Z^s."""
    s = len(xi)
    cols = [tuple(int(xi[a][j]) for a in range(s)) for j in range(len(xi[0]))]
    if rank(cols, s) != s:
        raise ValueError("Xi must have rank s")
    D, cosets, det_l = coset_structure(L)
    Linv = inverse(L)
    for c in cols:  # partition of unity on L needs L^{-1} Xi integer (Sec. 4.1)
        if any(sum(Linv[i][j] * c[j] for j in range(s)).denominator != 1 for i in range(s)):
            raise ValueError("L^{-1} Xi must be integer")
    fold = 2 if signed_permutation_invariant(xi) else 0
    return analyse_terms(name, L, box_spline_terms(xi, det_l), fold, [list(r) for r in xi], 0, anchor_den, verbose)


def analyse_voronoi(name, L, gens, order, anchor_den=64, verbose=False):
    """Run the analysis for phi = |det L| V_order on L Z^s, the Voronoi region of L being the
    centred zonotope of the generators gens (rational vectors).  The recorded direction matrix
    is 2 G (integers for the BCC and FCC regions)."""
    s = len(L)
    D, cosets, det_l = coset_structure(L)
    G = [[Fr(v) for v in g] for g in gens]
    if sum(t[2] for t in zonotope_tiling(G)) != det_l:
        raise ValueError("the zonotope's volume must be |det L| (a Voronoi region of L)")
    xi2 = [[int(2 * g[a]) for g in G] for a in range(s)]
    fold = 2 if signed_permutation_invariant(xi2) else 0
    return analyse_terms(name, L, voronoi_terms(G, order, det_l), fold, xi2, order, anchor_den, verbose)


def analyse_terms(name, L, terms, fold, xi_record, kind, anchor_den=64, verbose=False):
    """The analysis of Sec. 4 for phi = sum_t w_t M_{cols_t}(x + c_t) on the lattice L Z^s."""
    s = len(L)
    D, cosets, det_l = coset_structure(L)
    degree = len(terms[0].cols) - s
    if any(len(t.cols) - s != degree for t in terms):
        raise ValueError("all terms must have the same degree")

    # mesh plane normals and offsets (Sec. 3, the fine mesh Gamma) of every term
    offsets = {}
    term_normals = []
    for t in terms:
        dirs = sorted({_canon_dir(c) for c in t.cols})
        tn = set()
        for sub in itertools.combinations(dirs, s - 1):
            p = hyperplane_normal(list(sub), s)
            if p is not None:
                tn.add(p)
        tn = sorted(tn)
        term_normals.append(tn)
        for p in tn:
            sums = {Fr(0)}
            for c in t.cols:
                dv = sum(p[a] * c[a] for a in range(s))
                sums |= {x + dv for x in sums}
            pc = sum(p[a] * t.c[a] for a in range(s))
            offsets.setdefault(p, set()).update(x - pc for x in sums)
    normals = sorted(offsets)
    offsets = {p: sorted(v) for p, v in offsets.items()}

    # region of evaluation, folded
    half = Fr(D, 2)
    if fold == 2:
        chamber = [([-1 if k == s - 1 else 0 for k in range(s)], 0)]           # y_s >= 0
        chamber += [([1 if k == 0 else 0 for k in range(s)], half)]             # y_1 <= D/2
        for a in range(s - 1):                                                  # y_a >= y_{a+1}
            chamber.append(([(-1 if k == a else (1 if k == a + 1 else 0)) for k in range(s)], 0))
    else:
        chamber = []
        for a in range(s):
            chamber.append(([1 if k == a else 0 for k in range(s)], half))
            chamber.append(([-1 if k == a else 0 for k in range(s)], half))
    root = Cell(chamber, vertices(chamber, s))

    # planes p . y = e + D m (m integer) cutting the chamber interior
    planes = []
    for p in normals:
        vals = [sum(p[a] * v[a] for a in range(s)) for v in root.verts]
        lo, hi = min(vals), max(vals)
        for o in offsets[p]:
            k = math.floor((lo - o) / D)
            while o + D * k <= hi:
                e = o + D * k
                if lo < e < hi:
                    sg = [sum(p[a] * v[a] for a in range(s)) - e for v in root.verts]
                    if any(x > 0 for x in sg) and any(x < 0 for x in sg):
                        planes.append((p, e))
                k += 1
    planes = sorted(set(planes))

    cells = [root]
    for idx, (p, e) in enumerate(planes):
        nxt = []
        for c in cells:
            nxt.extend(split(c, p, e, s, idx))
        cells = nxt
    if verbose:
        print(f"{name}: s={s} terms={len(terms)} D={D} cosets={len(cosets)} fold={fold} Q={len(planes)} "
              f"cells={len(cells)}")

    # per term: support half-widths along its facet normals, support centre, bounding box
    geo = []
    for t, tn in zip(terms, term_normals):
        hw = {p: sum(abs(sum(p[a] * c[a] for a in range(s))) for c in t.cols) / 2 for p in tn}
        mid = [sum(c[a] for c in t.cols) / 2 - t.c[a] for a in range(s)]
        lo = [sum(min(0, c[a]) for c in t.cols) - t.c[a] for a in range(s)]
        hi = [sum(max(0, c[a]) for c in t.cols) - t.c[a] for a in range(s)]
        geo.append((tn, hw, mid, lo, hi))
    blo = [min(g[3][a] for g in geo) for a in range(s)]
    bhi = [max(g[4][a] for g in geo) for a in range(s)]
    groups = {}
    for ti, t in enumerate(terms):
        groups.setdefault(t.cols, []).append(ti)

    ctx = (s, D, terms, geo, groups, blo, bhi, anchor_den, len(planes))
    if len(terms) > 32 and len(cells) > 1:
        # many terms: the cells are independent, analyse them in worker processes
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(min(len(cells), os.cpu_count() or 1), mp_context=mp.get_context("fork"),
                                 initializer=_set_ctx, initargs=(ctx,)) as ex:
            pieces = list(ex.map(_cell_piece, cells))
    else:
        _set_ctx(ctx)
        pieces = [_cell_piece(c) for c in cells]

    codes = [pc.code for pc in pieces]
    Q = len(planes)
    sigma = _sigma_table(cells, chamber, planes, codes, s)
    r = 1 << Q
    halo = max((abs(g[a]) for pc in pieces for g in pc.sites for a in range(s)), default=0)
    lookups = max(len(pc.sites) for pc in pieces) * len(cosets)
    return SplineTables(name, s, [list(r_) for r_ in L], xi_record, det_l, D, cosets,
                        fold, degree, planes, r, sigma, pieces, halo, lookups, kind, smoothness(terms, s))


def smoothness(terms, s):
    """Continuity order k (phi in C^k) of a sum of box splines, the smallest over the terms: a box
    spline M_C is in C^(m-2), m the fewest columns whose removal leaves C not spanning R^s (the
    columns off some hyperplane spanned by columns of C) -- Sec. 3's smoothness of box splines."""
    best = None
    for t in terms:
        dirs = sorted({_canon_dir(c) for c in t.cols})
        m = None
        for sub in itertools.combinations(dirs, s - 1):
            p = hyperplane_normal(list(sub), s)
            if p is None:
                continue
            off = sum(1 for c in t.cols if sum(p[a] * c[a] for a in range(s)) != 0)
            m = off if m is None else min(m, off)
        k = m - 2
        best = k if best is None else min(best, k)
    return best


def sec42_compression(codes, Q):
    """Sec. 4.2's r: the smallest r with q mod r distinct over the cells' codes (brute force)."""
    return next(r for r in range(len(codes), (1 << Q) + 1) if len({q % r for q in codes}) == len(codes))


def _sigma_table(cells, chamber, planes, codes, s):
    """sigma[q] for every plane sign code q in [0, 2^Q).

    A query exactly on one or more planes (or where FP32 rounding flips a bit next to them) gets
    a code that no open cell has.  Any piece whose closure contains the query gives the right
    value (the spline is continuous), so such a code q is mapped through its closed region
    R_q = {y in the chamber : p_i . y >= e_i where bit i is set, <= e_i where it is not}: if R_q
    is not empty, to the first cell whose closure contains a relative-interior point of R_q
    (exact rational vertices); if it is empty, like the code at the smallest Hamming distance
    whose region is not.  This is why the kernels index sigma by q directly: Sec. 4.2's
    compression to q mod r keeps the cells' own codes apart but folds these codes onto
    unrelated pieces."""
    Q = len(planes)
    table = [-1] * (1 << Q)
    for j, q in enumerate(codes):
        table[q] = j
    if Q:
        import numpy as np
        from scipy.optimize import linprog
        A0 = [list(map(float, a)) for a, _ in chamber]
        b0 = [float(b) for _, b in chamber]
        for q in range(1 << Q):
            if table[q] >= 0:
                continue
            ineqs = list(chamber)
            for i, (p, e) in enumerate(planes):
                ineqs.append((list(p), e) if not (q >> i) & 1 else ([-x for x in p], -e))
            A = A0 + [list(map(float, a)) for a, _ in ineqs[len(chamber):]]
            b = b0 + [float(bb) for _, bb in ineqs[len(chamber):]]
            lp = linprog(np.zeros(s), A_ub=np.array(A), b_ub=np.array(b) + 1e-9, bounds=[(None, None)] * s,
                         method="highs")
            if lp.status != 0:
                continue
            vs = vertices(ineqs, s)
            if not vs:
                continue
            c = [sum(v[a] for v in vs) / len(vs) for a in range(s)]
            for j, cell in enumerate(cells):
                if all(sum(a[k] * c[k] for k in range(s)) <= bb for a, bb in cell.ineqs):
                    table[q] = j
                    break
    filled = [q for q in range(1 << Q) if table[q] >= 0]
    for q in range(1 << Q):
        if table[q] < 0:
            table[q] = table[min(filled, key=lambda f: (bin(q ^ f).count("1"), f))]
    return table


_CTX = None


def _set_ctx(ctx):
    global _CTX
    _CTX = ctx


def _cell_piece(c):
    """Stencil, exact polynomials and anchor of one cell (Sec. 4.1, the psi_j of S_j)."""
    s, D, terms, geo, groups, blo, bhi, anchor_den, Q = _CTX
    z = c.interior_point()
    # stencil: coset sites D g with z - D g in the open support of some term
    rng = [range(math.floor((z[a] - bhi[a]) / D), math.ceil((z[a] - blo[a]) / D) + 1) for a in range(s)]
    polys = {}
    for cols, tis in groups.items():
        per_site = []
        for g in itertools.product(*rng):
            w = [z[a] - D * g[a] for a in range(s)]
            hit = []
            for ti in tis:
                tn, hw, mid, _, _ = geo[ti]
                if all(abs(sum(p[a] * (w[a] - mid[a]) for a in range(s))) < hw[p] for p in tn):
                    hit.append(ti)
            if hit:
                per_site.append((g, [(terms[ti].w, terms[ti].c) for ti in hit]))
        if not per_site:
            continue
        for (g, _), P in zip(per_site, _piece_polynomials(cols, s, D, z, per_site)):
            polys[g] = polys[g].add(P) if g in polys else P
    sites = [list(g) for g in sorted(polys) if not polys[g].is_zero()]
    polys = [polys[tuple(g)] for g in sites]
    # expansion point: among the cell's vertices and its (dyadic-rounded) centroid, the one
    # that leaves the fewest nonzero coefficients (fewest FMAs), then the smallest ones
    cands = [list(v) for v in c.verts] + [[Fr(round(z[a] * anchor_den), anchor_den) for a in range(s)]]
    best = None
    for cand in cands:
        if any((2 * anchor_den * v).denominator != 1 for v in cand):
            continue                  # keep anchors exact in FP32
        shifted = [P.taylor_shift(cand) for P in polys]
        key = (sum(len(P.c) for P in shifted), max(abs(v) for P in shifted for v in P.c.values()))
        if best is None or key < best[0]:
            best = (key, cand, shifted)
    _, anchor, polys = best
    code = sum((c.signs[i] << i) for i in range(Q))
    return Piece(anchor, sites, polys, code, c.verts, c.ineqs)


def _piece_polynomials(cols, s, D, z, sites):
    """Exact polynomials of sum_t w_t M_cols(y - D g + c_t), y in the cell around the interior
    point z, for every entry (g, [(w_t, c_t), ...]) of sites (terms sharing the directions cols).

    M_{Xi'}(y + v) is computed by de Boor's recurrence on polynomials in y with t supported on a
    basis B of Xi' (t_xi = 0 off B), so (n'-s) M = sum_{xi in B} [M1 + t_xi (M0 - M1)]
    + sum_{xi not in B} M1 with M0 = M_{Xi'\\xi}(y + v), M1 = M_{Xi'\\xi}(y + v - xi).
    Memoised on (columns left, v), shared by all sites of the cell.
    """
    n = len(cols)
    memo = {}
    spans = {}
    basis_inv = {}
    bb = {}

    def spans_of(mask):
        if mask not in spans:
            vecs = [cols[j] for j in range(n) if mask >> j & 1]
            spans[mask] = len(vecs) >= s and rank(vecs, s) == s
        return spans[mask]

    def box(mask):
        if mask not in bb:
            lo = [sum(min(0, cols[j][a]) for j in range(n) if mask >> j & 1) for a in range(s)]
            hi = [sum(max(0, cols[j][a]) for j in range(n) if mask >> j & 1) for a in range(s)]
            bb[mask] = (lo, hi)
        return bb[mask]

    def basis(mask):
        if mask not in basis_inv:
            idx = [j for j in range(n) if mask >> j & 1]
            for sub in itertools.combinations(idx, s):
                B = [[cols[j][a] for j in sub] for a in range(s)]
                dB = det(B)
                if dB != 0:
                    basis_inv[mask] = (sub, inverse(B), dB)
                    break
        return basis_inv[mask]

    def M(mask, v):
        key = (mask, v)
        if key in memo:
            return memo[key]
        w = [z[a] + v[a] for a in range(s)]
        lo, hi = box(mask)
        if any(w[a] < lo[a] or w[a] > hi[a] for a in range(s)) or not spans_of(mask):
            memo[key] = Poly()
            return memo[key]
        cnt = bin(mask).count("1")
        sub, Binv, dB = basis(mask)
        if cnt == s:
            lam = [sum(Binv[i][a] * w[a] for a in range(s)) for i in range(s)]
            if any(l == 0 or l == 1 for l in lam):
                raise RuntimeError("interior point lies on a base-case facet")
            inside = all(0 < l < 1 for l in lam)
            memo[key] = Poly.const(Fr(1, abs(dB)) if inside else 0, s)
            return memo[key]
        acc = Poly()
        for j in range(n):
            if not mask >> j & 1:
                continue
            rest = mask & ~(1 << j)
            if not spans_of(rest):
                continue
            v1 = tuple(v[a] - cols[j][a] for a in range(s))
            M1 = M(rest, v1)
            if j in sub:
                i = sub.index(j)
                # t_j(y) = sum_a Binv[i][a] (y_a + v_a)
                aff = [sum(Binv[i][a] * v[a] for a in range(s))] + [Binv[i][a] for a in range(s)]
                M0 = M(rest, v)
                diff = M0.add(M1, -1)
                acc = acc.add(M1).add(diff.mul_affine(aff))
            else:
                acc = acc.add(M1)
        res = acc.scale(Fr(1, cnt - s))
        memo[key] = res
        return res

    full = (1 << n) - 1
    out = []
    for g, wcs in sites:
        acc = Poly()
        for w, c in wcs:
            v = tuple(Fr(c[a]) - D * g[a] for a in range(s))
            acc = acc.add(M(full, v).scale(w))
        out.append(acc)
    return out
