"""Exact rational twin of the box-spline oracle, for tiny inputs.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only tests/ use it; the CUDA path never
imports it.

It evaluates the same definition as ``boxspline_oracle.c`` -- the box spline M_Xi of Sec. 3 by
de Boor's recurrence, (n - s) M_Xi(x) = sum_xi [t_xi M_{Xi minus xi}(x) + (1 - t_xi)
M_{Xi minus xi}(x - xi)] for any t with Xi t = x, with the base case 1/|det Z| on Z[0,1)^s and
the terms whose remaining directions do not span R^s dropped -- but with Python fractions
throughout (t = Xi^T (Xi Xi^T)^-1 x, exact), so its values at rational points are exact.  FP32
query points are dyadic rationals, so the FP64 oracle can be checked against it to its rounding
error.  phi(x) = |det L| M_Xi(x + sum(Xi)/2), as the FP64 oracle.
"""
from __future__ import annotations

from fractions import Fraction as Fr
from functools import lru_cache


def _det(m):
    """Determinant of a square matrix of fractions (Gaussian elimination, exact)."""
    a = [list(r) for r in m]
    n = len(a)
    det = Fr(1)
    for c in range(n):
        p = next((r for r in range(c, n) if a[r][c] != 0), None)
        if p is None:
            return Fr(0)
        if p != c:
            a[c], a[p] = a[p], a[c]
            det = -det
        det *= a[c][c]
        for r in range(c + 1, n):
            f = a[r][c] / a[c][c]
            if f:
                for k in range(c, n):
                    a[r][k] -= f * a[c][k]
    return det


def _solve(m, b):
    """m y = b for a nonsingular square matrix of fractions."""
    n = len(m)
    a = [list(m[r]) + [b[r]] for r in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[p] = a[p], a[c]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c] / a[c][c]
                for k in range(c, n + 1):
                    a[r][k] -= f * a[c][k]
    return [a[r][n] / a[r][r] for r in range(n)]


def _rank(m):
    a = [list(r) for r in m]
    rows, cols = len(a), len(a[0]) if a else 0
    rank = 0
    for c in range(cols):
        p = next((r for r in range(rank, rows) if a[r][c] != 0), None)
        if p is None:
            continue
        a[rank], a[p] = a[p], a[rank]
        for r in range(rows):
            if r != rank and a[r][c] != 0:
                f = a[r][c] / a[rank][c]
                for k in range(c, cols):
                    a[r][k] -= f * a[rank][k]
        rank += 1
    return rank


class ExactBoxSpline:
    """M_Xi and phi in exact rational arithmetic.  xi: s x n integer direction matrix (nested
    lists or an array), det_l: |det L| of the lattice."""

    def __init__(self, xi, det_l: int):
        self.s = len(xi)
        self.n = len(xi[0])
        self.cols = [tuple(Fr(int(xi[a][j])) for a in range(self.s)) for j in range(self.n)]
        self.det_l = Fr(det_l)
        self.centre = tuple(sum(c[a] for c in self.cols) / 2 for a in range(self.s))
        self._M = lru_cache(maxsize=None)(self._M_uncached)

    def _M_uncached(self, idx: tuple, x: tuple) -> Fr:
        s = self.s
        Z = [[self.cols[j][a] for j in idx] for a in range(s)]          # s x m
        m = len(idx)
        if _rank(Z) < s:
            return Fr(0)                       # a singular measure: zero off its plane
        if m == s:
            d = _det(Z)
            y = _solve(Z, list(x))
            inside = all(Fr(0) <= v < Fr(1) for v in y)
            return Fr(1) / abs(d) if inside else Fr(0)
        # t = Z^T (Z Z^T)^-1 x solves Z t = x
        ZZt = [[sum(Z[a][k] * Z[b][k] for k in range(m)) for b in range(s)] for a in range(s)]
        w = _solve(ZZt, list(x))
        t = [sum(Z[a][k] * w[a] for a in range(s)) for k in range(m)]
        acc = Fr(0)
        for k in range(m):
            rest = idx[:k] + idx[k + 1:]
            xi = self.cols[idx[k]]
            shifted = tuple(x[a] - xi[a] for a in range(s))
            acc += t[k] * self._M(rest, x) + (1 - t[k]) * self._M(rest, shifted)
        return acc / (m - s)

    def M(self, x) -> Fr:
        return self._M(tuple(range(self.n)), tuple(Fr(v) for v in x))

    def phi(self, z) -> Fr:
        """|det L| M_Xi(z + sum(Xi)/2) at a point z (floats are taken exactly)."""
        return self.det_l * self.M(tuple(Fr(v) + c for v, c in zip(z, self.centre)))
