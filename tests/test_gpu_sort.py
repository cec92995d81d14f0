"""Spatial sort of queries (Morton-ordered bins) and the adjoint on sorted queries, which sums in
shared memory: a valid permutation, keys in order, and the adjoint still equal to the oracle's."""
import numpy as np
import pytest

import oracle
from synth import interior_box, make_rng, uniform_points

from _gpu_common import mixed_points, require_cuda, spline_setup

pytestmark = pytest.mark.gpu


def _morton(bins, bits=10):
    key = np.zeros(len(bins), dtype=np.int64)
    s = bins.shape[1]
    for b in range(bits):
        for a in range(s):
            key |= ((bins[:, a] >> b) & 1) << (b * s + a)
    return key


@pytest.mark.parametrize("name,n_axis", [("bcc_quintic", 20), ("cc_7dir", 24), ("d4s_8dir", 8)])
def test_sort_points_is_a_spatial_permutation(name, n_axis):
    torch = require_cuda()
    from paper_2102_08514_b300.binding import Interpolator
    sp, lat, xi, detl = spline_setup(name)
    s = xi.shape[0]
    dims = (n_axis,) * s
    itp = Interpolator(np.asarray(lat.L), xi, dims, "f32")
    lo, hi = interior_box(name, dims)
    pts = uniform_points(make_rng(81, 0), 50_000, lo, hi)
    perm, srt = itp.sort_points(torch.from_numpy(pts).cuda())
    perm = perm.cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(len(pts)))
    assert np.array_equal(srt.cpu().numpy(), pts[perm])
    # keys: Morton order of the coset-0 cell (padded) divided into bins of 2^bb cells
    bb = 2 if s == 3 else 1
    cell = np.floor(pts[perm].astype(np.float64) / lat.D + 0.5).astype(np.int64) + 2 * itp.info.halo
    key = _morton(cell >> bb)
    assert np.all(np.diff(key) >= 0)


@pytest.mark.parametrize("name,n_axis", [("bcc_quintic", 16), ("fcc_6dir", 14), ("cc_7dir", 18)])
def test_adjoint_on_sorted_queries_matches_oracle(name, n_axis):
    torch = require_cuda()
    from paper_2102_08514_b300.binding import Interpolator
    sp, lat, xi, detl = spline_setup(name)
    dims = (n_axis,) * xi.shape[0]
    itp = Interpolator(np.asarray(lat.L), xi, dims, "f32")
    pts = torch.from_numpy(mixed_points(name, dims, 8_000, 82)).cuda()
    g = torch.from_numpy(make_rng(83, 0).uniform(-1, 1, pts.shape[0]).astype(np.float32)).cuda()
    perm, srt = itp.sort_points(pts)
    gs = g[perm.long()]
    d_sorted, _ = itp.backward(srt, gs)
    d_plain, _ = itp.backward(pts, g)
    shape = itp.shape
    o = oracle.Spline(xi, detl)
    P = srt.cpu().numpy().astype(np.float64)
    ref = oracle.adjoint(o, lat.D, lat.cosets, shape, P, gs.cpu().numpy().astype(np.float64))
    bound = oracle.adjoint(o, lat.D, lat.cosets, shape, P, np.abs(gs.cpu().numpy()).astype(np.float64))
    tol = 4e-6 * bound + 1e-7
    assert np.all(np.abs(d_sorted.cpu().numpy() - ref) <= tol)
    assert np.all(np.abs(d_plain.cpu().numpy() - ref) <= tol)
