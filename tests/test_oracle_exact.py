"""The FP64 oracle against its exact rational twin (oracle/exact.py: the same recurrence in Python
fractions) at FP32-representable points, i.e. dyadic rationals, where the twin's values are
exact: a wrong sign, index or weight in the C recurrence shows far above its rounding."""
import numpy as np
import pytest

import oracle
from oracle.exact import ExactBoxSpline
from synth import LATTICES, SPLINES


def _points(name, n, seed):
    rng = np.random.default_rng(seed)
    sp = SPLINES[name]
    xi = np.asarray(sp.xi)
    hw = np.abs(xi).sum(axis=1) / 2.0                 # half-widths of the support's bounding box
    return (rng.uniform(-hw, hw, (n, xi.shape[0]))).astype(np.float32)


@pytest.mark.parametrize("name,n", [("bcc_linear", 12), ("bcc_quintic", 6), ("fcc_6dir", 10), ("cc_7dir", 6),
                                    ("bcc_quartic", 6), ("cc_voronoi1", 8)])
def test_fp64_oracle_equals_exact_recurrence(name, n):
    sp = SPLINES[name]
    lat = LATTICES[sp.lattice]
    xi = np.asarray(sp.xi)
    detl = abs(round(np.linalg.det(np.asarray(lat.L, dtype=float))))
    exact = ExactBoxSpline(xi.tolist(), detl)
    o = oracle.Spline(xi, detl)
    pts = _points(name, n, 11)
    got = o.phi(pts.astype(np.float64))
    ref = np.array([float(exact.phi(p.tolist())) for p in pts])
    assert np.count_nonzero(ref) >= 3
    assert np.abs(got - ref).max() <= 1e-15 * max(1.0, np.abs(ref).max()), np.abs(got - ref).max()


def test_exact_twin_closed_forms():
    # the twin on its own: a 1-D cardinal B-spline of order 3 and the bilinear hat (Xi = I, I)
    quad = ExactBoxSpline([[1, 1, 1]], 1)
    from fractions import Fraction as Fr
    # centred quadratic B-spline: 3/4 - x^2 on |x| < 1/2, (3/2 - |x|)^2 / 2 on 1/2 <= |x| < 3/2
    for x in (Fr(0), Fr(1, 4), Fr(3, 4), Fr(-5, 4), Fr(2)):
        ax = abs(x)
        want = Fr(3, 4) - x * x if ax < Fr(1, 2) else ((Fr(3, 2) - ax) ** 2 / 2 if ax < Fr(3, 2) else Fr(0))
        assert quad.phi([x]) == want
    hat = ExactBoxSpline([[1, 0, 1, 0], [0, 1, 0, 1]], 1)
    for x, y in ((Fr(1, 3), Fr(-1, 2)), (Fr(0), Fr(0)), (Fr(7, 8), Fr(1, 8))):
        assert hat.phi([x, y]) == max(Fr(0), 1 - abs(x)) * max(Fr(0), 1 - abs(y))
