"""ctypes front end of the FP64 CPU oracle (``boxspline_oracle.c``).

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import this module.  The CUDA product path never imports,
links or runs anything under ``oracle/``; the two share no code.

What it computes (Horacsek & Alim, arXiv 2102.08514):

* ``Spline.M``      -- the box spline M_Xi of Sec. 3 (base case 1/|det Xi| on Xi[0,1)^s, support the
  zonotope), by de Boor's recurrence with exact decisions (see the C file's header).
* ``Spline.phi``    -- the centred, normalised basis phi(x) = |det L| M_Xi(x + sum(Xi)/2), so that
  phi has partition of unity on L Z^s (Sec. 4.1 requires it).
* ``eval_sum``      -- the convolution sum of Eq. 1 (h = 1) split over the Cartesian cosets of
  Sec. 4.1, f(x) = sum_k sum_i c_k[i] phi(x - D i - l_k), summed by brute force; optional grad.
* ``adjoint``       -- dL/dc_k[i] = sum_q g_q phi(x_q - D i - l_k).
* ``cells``         -- the exact shift rho to the region of evaluation (Sec. 4.1), here the cube
  [-D/2, D/2)^s centred on the nearest site of each coset.
* ``VoronoiSpline`` -- the Voronoi splines V_n of Sec. 3 (the Voronoi region's indicator convolved
  with itself), as the sum of shifted box splines Sec. 3 describes, each by the box-spline oracle;
  its ``eval_sum`` / ``adjoint`` / ``phi`` mirror the functions above.
* ``prefilter``     -- a discrete filter on the lattice (Sec. 5.2's quasi-interpolation prefilter
  for the D4 spline: ``d4_quasi_interpolation_taps``), computed on the world grid.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from itertools import combinations, combinations_with_replacement, product
from math import factorial

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "boxspline_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (gcc, OpenMP); rebuilt when the
    source's hash differs from the one recorded beside the library."""
    with open(_SRC, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    stamp = _LIB + ".stamp"
    current = os.path.exists(_LIB) and os.path.exists(stamp) and open(stamp).read().strip() == digest
    if force or not current:
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(digest)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_void_p)]
        lib.orc_destroy.argtypes = [P]
        lib.orc_M.argtypes = [P, ctypes.c_uint, I64, P, P]
        lib.orc_phi.argtypes = [P, I64, P, P, P]
        lib.orc_eval.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, I64, P, P, P, ctypes.c_int]
        lib.orc_adjoint.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, I64, P, P, P]
        lib.orc_cells.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, I64, P, P, P]
        for f in (lib.orc_create, lib.orc_M, lib.orc_phi, lib.orc_eval, lib.orc_adjoint, lib.orc_cells):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}"
                           + (" (point not exactly representable)" if rc == 2 else ""))


class Spline:
    """A box spline M_Xi (columns of ``xi`` are the directions) and its centred basis phi.

    ``det_l`` is |det L| of the lattice phi is used on; ``tmode`` picks the solution t of Xi t = x
    used by the recurrence (0: minimum norm, 1: supported on a basis) -- both are valid, which is
    what the two-t agreement test checks.
    """

    def __init__(self, xi, det_l: float = 1.0, tmode: int = 0):
        xi = np.asarray(xi, dtype=np.int64)
        if xi.ndim != 2:
            raise ValueError("xi must be an s x n integer matrix")
        self.xi = xi
        self.s, self.n = xi.shape
        self.det_l = float(det_l)
        cols = np.ascontiguousarray(xi.T, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(_load().orc_create(self.s, self.n, _ptr(cols), self.det_l, tmode, ctypes.byref(h)),
               "create")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    @property
    def halfwidth(self) -> np.ndarray:
        return np.abs(self.xi).sum(axis=1) / 2.0

    def M(self, w, mask: int | None = None) -> np.ndarray:
        """Raw M_{Xi_mask}(w) (uncentred, integral 1); mask defaults to all columns."""
        w = np.ascontiguousarray(np.atleast_2d(np.asarray(w, dtype=np.float64)))
        out = np.empty(w.shape[0])
        m = (1 << self.n) - 1 if mask is None else mask
        _check(_load().orc_M(self._h, m, w.shape[0], _ptr(w), _ptr(out)), "M")
        return out

    def phi(self, z, grad: bool = False):
        z = np.ascontiguousarray(np.atleast_2d(np.asarray(z, dtype=np.float64)))
        out = np.empty(z.shape[0])
        g = np.empty_like(z) if grad else None
        _check(_load().orc_phi(self._h, z.shape[0], _ptr(z), _ptr(out), _ptr(g)), "phi")
        return (out, g) if grad else out


def lattice_sites(L, lo, hi) -> np.ndarray:
    """All points of L Z^s inside the box [lo, hi] (integer L), by a membership test on Z^s:
    z is a site iff adj(L) z = 0 mod det L.  Independent of any coset decomposition."""
    L = np.asarray(L, dtype=np.int64)
    s = L.shape[0]
    det = int(round(np.linalg.det(L)))
    adj = np.round(np.linalg.inv(L) * det).astype(np.int64)
    rng = [range(int(np.ceil(lo[a])), int(np.floor(hi[a])) + 1) for a in range(s)]
    pts = np.array(list(product(*rng)), dtype=np.int64).reshape(-1, s)
    keep = np.all((pts @ adj.T) % abs(det) == 0, axis=1)
    return pts[keep]


def eval_sum(spline: Spline, D: int, cosets, coeffs, points, grad: bool = False, nthreads: int = 0):
    """f(x_q) = sum_k sum_i c_k[i] phi(x_q - D i - l_k) (and grad f) in FP64, brute force.

    ``coeffs`` has shape (M, N_1, ..., N_s) (coset-major, last axis fastest); points (Q, s).
    Outside the stored arrays the coefficients are taken as 0.
    """
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    lk = np.ascontiguousarray(cosets, dtype=np.int32).reshape(-1, spline.s)
    dims = np.ascontiguousarray(c.shape[1:], dtype=np.int32)
    p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, spline.s)
    out = np.empty(p.shape[0])
    g = np.empty_like(p) if grad else None
    _check(_load().orc_eval(spline._h, D, lk.shape[0], _ptr(lk), _ptr(dims), _ptr(c), p.shape[0],
                            _ptr(p), _ptr(out), _ptr(g), nthreads), "eval")
    return (out, g) if grad else out


def adjoint(spline: Spline, D: int, cosets, shape, points, g) -> np.ndarray:
    """dL/dc for dL/df = g: sum_q g_q phi(x_q - D i - l_k), in the coefficient layout ``shape``."""
    lk = np.ascontiguousarray(cosets, dtype=np.int32).reshape(-1, spline.s)
    dims = np.ascontiguousarray(shape[1:], dtype=np.int32)
    p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, spline.s)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    d = np.zeros(shape, dtype=np.float64)
    _check(_load().orc_adjoint(spline._h, D, lk.shape[0], _ptr(lk), _ptr(dims), p.shape[0], _ptr(p),
                               _ptr(gg), _ptr(d)), "adjoint")
    return d


def cells(s: int, D: int, cosets, points):
    """Exact nearest coset site i (Q, M, s) int32 and offset y = x - l_k - D i (Q, M, s)."""
    lk = np.ascontiguousarray(cosets, dtype=np.int32).reshape(-1, s)
    p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, s)
    q, m = p.shape[0], lk.shape[0]
    ci = np.empty((q, m, s), dtype=np.int32)
    off = np.empty((q, m, s), dtype=np.float64)
    _check(_load().orc_cells(s, D, m, _ptr(lk), q, _ptr(p), _ptr(ci), _ptr(off)), "cells")
    return ci, off


def folded_offsets(offsets: np.ndarray) -> np.ndarray:
    """Fold offsets into the chamber D/2 >= y_1 >= ... >= y_s >= 0 of the signed permutations
    (the reflection of Sec. 4.2 generalised to the full symmetry group of the cube)."""
    return -np.sort(-np.abs(offsets), axis=-1)


# ----------------------------------------------------------------------------- Voronoi splines

def _det3(m):
    from fractions import Fraction as Fr
    if len(m) == 1:
        return Fr(m[0][0])
    return sum((-1) ** j * m[0][j] * _det3([r[:j] + r[j + 1:] for r in m[1:]]) for j in range(len(m)))


def _solve_exact(A, b):
    """Cramer's rule over Fractions (A small and nonsingular)."""
    d = _det3(A)
    out = []
    for j in range(len(A)):
        Aj = [row[:j] + [b[i]] + row[j + 1:] for i, row in enumerate(A)]
        out.append(_det3(Aj) / d)
    return out


def zonotope_tiles(gens, heights):
    """Parallelepiped tiling of Z(G) = sum_j [0, g_j]: for every basis B of G, the offset z_B with
    z_B + B[0,1)^s a tile.  It is the regular tiling of the heights h (one per generator, generic):
    the tile of B projects the lower facet of the lifted zonotope spanned by the (g_b, h_b), which
    contains the lifted g_j (j not in B) lying below the affine function through B's lifts.
    Returns [(B, z_B, |det B|)]."""
    from fractions import Fraction as Fr
    s = len(gens[0])
    out = []
    for B in combinations(range(len(gens)), s):
        rows = [[Fr(gens[b][a]) for a in range(s)] for b in B]       # g_b as rows
        dB = _det3(rows)
        if dB == 0:
            continue
        a_ = _solve_exact(rows, [Fr(heights[b]) for b in B])          # a . g_b = h_b
        z = [Fr(0)] * s
        for j, g in enumerate(gens):
            if j in B:
                continue
            below = Fr(heights[j]) - sum(a_[k] * g[k] for k in range(s))
            if below == 0:
                raise ValueError("heights are not generic")
            if below < 0:
                z = [z[k] + g[k] for k in range(s)]
        out.append((B, tuple(z), abs(dB)))
    return out


class VoronoiSpline:
    """phi = |det L| V_n on the lattice L, with V_0 = chi (1/|det L| on the Voronoi region, here the
    centred zonotope of the generators G) and V_n = V_0 * V_{n-1} (Sec. 3).

    Following Sec. 3, V_0 is rewritten as a sum of constant box splines (the tiles z_B + B[0,1)^s of
    the zonotope, each |det B| M_B), and the (n+1)-fold convolution is expanded by the multinomial
    theorem; a convolution of box splines is the box spline of the concatenated directions,
    shifted by the sum of the shifts.  Each term w M_{C}(x + c) is evaluated by the box-spline
    oracle with the directions doubled (G is half-integral): M_C(y) = 2^s M_{2C}(2 y).
    ``heights`` picks the tiling (any generic choice gives the same V_n).
    """

    def __init__(self, L, gens, order: int, heights=None):
        from fractions import Fraction as Fr
        L = np.asarray(L, dtype=np.int64)
        self.s = L.shape[0]
        self.det_l = abs(int(round(np.linalg.det(L))))
        self.gens = [tuple(Fr(v) for v in g) for g in gens]
        self.order = order
        if heights is None:
            heights = [Fr(2 * j * j + 3 * j + 5, 7 + j) for j in range(len(self.gens))]
        self.tiles = zonotope_tiles(self.gens, heights)
        s = self.s
        ctr = [sum(g[a] for g in self.gens) / 2 for a in range(s)]
        terms = {}
        for combo in combinations_with_replacement(range(len(self.tiles)), order + 1):
            mult = factorial(order + 1)
            for i in set(combo):
                mult //= factorial(combo.count(i))
            w = Fr(mult) / Fr(self.det_l) ** order
            for i in combo:
                w *= self.tiles[i][2]
            dirs = tuple(sorted(tuple(int(2 * v) for v in self.gens[b]) for i in combo for b in self.tiles[i][0]))
            shift = tuple(sum(ctr[a] - self.tiles[i][1][a] for i in combo) for a in range(s))
            terms[(dirs, shift)] = terms.get((dirs, shift), 0) + w
        # group by direction multiset: one oracle Spline per group, (weight, doubled shift) list
        self.groups = {}
        for (dirs, shift), w in sorted(terms.items()):
            xi2 = np.array(dirs, dtype=np.int64).T
            # M_C(x + c) = 2^s M_{2C}(2x + 2c); the Spline is centred, so pass 2x + 2c - sum(2C)/2
            d2 = np.array([float(2 * shift[a]) for a in range(s)]) - xi2.sum(axis=1) / 2.0
            self.groups.setdefault(dirs, []).append((float(w) * 2 ** s, d2))
        self.n_terms = len(terms)
        self._splines = {dirs: Spline(np.array(dirs, dtype=np.int64).T, 1.0) for dirs in self.groups}

    @property
    def halfwidth(self) -> np.ndarray:
        """Half-widths of the support's bounding box: (n+1) times the Voronoi region's."""
        return (self.order + 1) * np.array([sum(abs(float(g[a])) for g in self.gens) / 2 for a in range(self.s)])

    def phi(self, z, grad: bool = False):
        """phi(z) (and grad) at points z (Q, s)."""
        z = np.atleast_2d(np.asarray(z, dtype=np.float64))
        out = np.zeros(z.shape[0])
        g = np.zeros_like(z) if grad else None
        for dirs, ws in self.groups.items():
            sp = self._splines[dirs]
            for w, d2 in ws:
                r = sp.phi(2.0 * z + d2, grad=grad)
                if grad:
                    out += w * r[0]
                    g += 2.0 * w * r[1]
                else:
                    out += w * r
        return (out, g) if grad else out

    def eval_sum(self, D: int, cosets, coeffs, points, grad: bool = False, nthreads: int = 0):
        """f(x_q) = sum_k sum_i c_k[i] phi(x_q - D i - l_k) (and grad f) in FP64, brute force."""
        p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, self.s)
        lk2 = 2 * np.asarray(cosets, dtype=np.int64).reshape(-1, self.s)
        out = np.zeros(p.shape[0])
        g = np.zeros_like(p) if grad else None
        for dirs, ws in self.groups.items():
            sp = self._splines[dirs]
            for w, d2 in ws:
                r = eval_sum(sp, 2 * D, lk2, coeffs, 2.0 * p + d2, grad=grad, nthreads=nthreads)
                if grad:
                    out += w * r[0]
                    g += 2.0 * w * r[1]
                else:
                    out += w * r
        return (out, g) if grad else out

    def adjoint(self, D: int, cosets, shape, points, g) -> np.ndarray:
        """dL/dc for dL/df = g: sum_q g_q phi(x_q - D i - l_k)."""
        p = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, self.s)
        lk2 = 2 * np.asarray(cosets, dtype=np.int64).reshape(-1, self.s)
        d = np.zeros(shape)
        for dirs, ws in self.groups.items():
            sp = self._splines[dirs]
            for w, d2 in ws:
                d += w * adjoint(sp, 2 * D, lk2, shape, 2.0 * p + d2, g)
        return d


# ----------------------------------------------------------------------------- lattice prefilter

def prefilter(L, D: int, cosets, samples, taps, weights) -> np.ndarray:
    """c(n) = sum_t w_t f(n + v_t) at every stored site n (the quasi-interpolation prefilter of
    Sec. 5.2 is 7/3 at v = 0 and -1/18 at the 24 sites at distance sqrt(2)), with f the samples
    at the stored sites and 0 elsewhere.

    Computed on the world grid, without any coset arithmetic: the samples are placed at their
    world positions D i + l_k of a dense array (zero at non-sites), the filter is the weighted
    sum of copies of that array shifted by the taps, read back at the sites.  The taps must be
    lattice vectors (checked by the membership test adj(L) v = 0 mod det L)."""
    L = np.asarray(L, dtype=np.int64)
    f = np.asarray(samples, dtype=np.float64)
    s = L.shape[0]
    taps = np.asarray(taps, dtype=np.int64).reshape(-1, s)
    det = int(round(np.linalg.det(L)))
    adj = np.round(np.linalg.inv(L) * det).astype(np.int64)
    if np.any((taps @ adj.T) % abs(det) != 0):
        raise ValueError("filter taps must be lattice vectors")
    dims = f.shape[1:]
    R = int(np.abs(taps).max()) if taps.size else 0
    W = np.zeros(tuple(D * n + 2 * R for n in dims))
    for k, lk in enumerate(np.asarray(cosets, dtype=np.int64).reshape(-1, s)):
        W[tuple(slice(R + lk[a], R + lk[a] + D * dims[a], D) for a in range(s))] = f[k]
    C = np.zeros_like(W)
    for v, w in zip(taps, weights):
        # C[x] += w W[x + v] wherever x + v lies in the array
        dst = tuple(slice(max(0, -v[a]), W.shape[a] - max(0, v[a])) for a in range(s))
        src = tuple(slice(max(0, v[a]), W.shape[a] - max(0, -v[a])) for a in range(s))
        C[dst] += float(w) * W[src]
    out = np.empty_like(f)
    for k, lk in enumerate(np.asarray(cosets, dtype=np.int64).reshape(-1, s)):
        out[k] = C[tuple(slice(R + lk[a], R + lk[a] + D * dims[a], D) for a in range(s))]
    return out


def d4_quasi_interpolation_taps():
    """Sec. 5.2: 7/3 at the origin and -1/18 at the 24 D4 sites at distance sqrt(2), the vectors
    with two entries +-1 and two zeros."""
    taps, w = [(0, 0, 0, 0)], [7.0 / 3.0]
    for a in range(4):
        for b in range(a + 1, 4):
            for sa in (1, -1):
                for sb in (1, -1):
                    v = [0, 0, 0, 0]
                    v[a], v[b] = sa, sb
                    taps.append(tuple(v))
                    w.append(-1.0 / 18.0)
    return np.array(taps, dtype=np.int32), np.array(w)
