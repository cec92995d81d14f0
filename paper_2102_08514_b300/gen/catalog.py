"""Built-in (lattice, direction matrix) pairs, in the paper's integer frame.

Lattice generating matrices are those of Sec. 3 (L_BCC, L_FCC) and the D4* lattice
Z^4 u (Z^4 + (1/2,1/2,1/2,1/2)) scaled by 2 so that it is an integer lattice (all coordinates of
equal parity).  Direction matrices are the Table 1 rows of Sec. 5.1 and the 8-direction D4 spline
of Sec. 5.2 (its sign convention is immaterial once the spline is centred).

Voronoi splines (Sec. 3, V_n = chi * V_{n-1}, Table 1's BCC and FCC Voronoi splines on their own
lattices) are given by their lattice, the generators G of the Voronoi region as a centred
zonotope sum_j [-g_j/2, g_j/2], and the order n:
  BCC (integer frame, |det L| = 4): the truncated octahedron |y_a| <= 1, |y_1|+|y_2|+|y_3| <= 3/2,
      the zonotope of the six vectors (+-1/2, +-1/2, 0) up to permutation and sign;
  FCC (|det L| = 2): the rhombic dodecahedron |y_a| + |y_b| <= 1, the zonotope of the four
      body diagonals (+-1/2, +-1/2, +-1/2).
"""
from __future__ import annotations

from fractions import Fraction

L_CC = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
L_BCC = [[-1, 1, 1], [1, -1, 1], [1, 1, -1]]          # Sec. 3
L_FCC = [[0, 1, 1], [1, 0, 1], [1, 1, 0]]             # Sec. 3
L_D4S = [[2, 0, 0, 1], [0, 2, 0, 1], [0, 0, 2, 1], [0, 0, 0, 1]]  # 2Z^4 u 2Z^4+(1,1,1,1)
L_D4 = [[-1, 0, 0, 0], [1, 0, -1, -1], [0, -1, 0, 1], [0, -1, 1, 0]]  # Sec. 5.2: even coordinate sum

XI_BCC_RD = [[-1, 1, 1, -1], [1, -1, 1, -1], [1, 1, -1, -1]]      # Table 1, linear RD
XI_FCC6 = [[1, -1, 1, 1, 0, 0], [1, 1, 0, 0, 1, -1], [0, 0, 1, -1, 1, 1]]   # Table 1, FCC 6-dir
XI_CC7 = [[1, 0, 0, -1, 1, 1, -1], [0, 1, 0, 1, -1, 1, -1], [0, 0, 1, 1, 1, -1, -1]]  # Table 1, TRD
XI_BCC_QUARTIC = [[2, 0, 0, -1, 1, 1, -1], [0, 2, 0, 1, -1, 1, -1], [0, 0, 2, 1, 1, -1, -1]]
XI_D4 = [[1, 1, 1, 1, 1, 1, 1, 1],
         [1, 1, 1, 1, -1, -1, -1, -1],
         [1, 1, -1, -1, 1, 1, -1, -1],
         [1, -1, 1, -1, 1, -1, 1, -1]]                # Sec. 5.2, 8 directions (1, +-1, +-1, +-1)


def _twice(xi):
    return [row + row for row in xi]


XI_I3 = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]


def _repeat(xi, k):
    return [row * k for row in xi]


CATALOG = {
    "bcc_linear": (L_BCC, XI_BCC_RD),
    "bcc_quintic": (L_BCC, _twice(XI_BCC_RD)),
    "fcc_6dir": (L_FCC, XI_FCC6),
    "cc_7dir": (L_CC, XI_CC7),
    "d4s_8dir": (L_D4S, XI_D4),
    "d4_8dir": (L_D4, XI_D4),                       # Sec. 5.2: the same spline on D4 (8 cosets)
    # the other Table 1 box splines
    "bcc_quartic": (L_BCC, XI_BCC_QUARTIC),        # quartic truncated rhombic dodecahedron on BCC
    "cc_linear_rd": (L_CC, XI_BCC_RD),             # linear rhombic dodecahedron on CC
    "cc_voronoi1": (L_CC, _repeat(XI_I3, 2)),      # CC Voronoi spline 1 = trilinear B-spline
    "cc_voronoi2": (L_CC, _repeat(XI_I3, 3)),      # CC Voronoi spline 2 = triquadratic B-spline
    "cc_voronoi3": (L_CC, _repeat(XI_I3, 4)),      # CC Voronoi spline 3 = tricubic B-spline
}


_H = Fraction(1, 2)
G_BCC_VORONOI = [(_H, _H, 0), (_H, -_H, 0), (_H, 0, _H), (_H, 0, -_H), (0, _H, _H), (0, _H, -_H)]
G_FCC_VORONOI = [(_H, _H, _H), (_H, -_H, -_H), (-_H, _H, -_H), (-_H, -_H, _H)]

VORONOI = {
    "bcc_voronoi1": (L_BCC, G_BCC_VORONOI, 1),
    "fcc_voronoi1": (L_FCC, G_FCC_VORONOI, 1),
    "fcc_voronoi2": (L_FCC, G_FCC_VORONOI, 2),
    "bcc_voronoi2": (L_BCC, G_BCC_VORONOI, 2),
}


def catalog_entry(name: str):
    L, xi = CATALOG[name]
    return [list(r) for r in L], [list(r) for r in xi]
