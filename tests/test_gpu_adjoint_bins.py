"""The adjoint on spatially binned queries (interp_backward's counting sort into bins of coset
cells, shared-memory boxes per bin) against the FP64 oracle's brute-force adjoint and against the
unbinned scatter.

Tolerance as for every adjoint test: per coefficient <= 4e-6 * sum_q |g_q| phi(x_q - n) + 1e-7
(FP32 contributions summed in an order that varies between runs)."""
import numpy as np
import pytest

from synth import LATTICES, SPLINES, WORKLOADS, coefficients, interior_box, make_rng, uniform_points

from _gpu_common import OracleSpline, make_interpolator, mixed_points, require_cuda, spline_setup

pytestmark = pytest.mark.gpu

# the 3-D splines with fewer than 4 pieces (the ones the binned adjoint serves), small cases
CASES = {"bcc_linear": (12, 4133), "bcc_quintic": (12, 2085), "fcc_6dir": (10, 3011), "cc_7dir": (14, 2107),
         "bcc_quartic": (12, 2091), "cc_voronoi3": (12, 389)}


def _adjoint(itp, pts, g, bins):
    import torch
    itp.set_option("adjoint_bins", bins)
    dc = torch.zeros(itp.shape, device="cuda")
    itp.backward(pts, g, dc)
    torch.cuda.synchronize()
    return dc


@pytest.mark.parametrize("name", list(CASES))
def test_binned_adjoint_matches_oracle(name):
    # mixed points: interior, a band around the data (partly out of range), exact ties, NaN/inf,
    # far away; some gout are zero
    torch = require_cuda()
    n_axis, nq = CASES[name]
    sp, lat, xi, detl = spline_setup(name)
    dims = (n_axis,) * 3
    itp = make_interpolator(name, dims)
    pts = mixed_points(name, dims, nq, 31)
    g = make_rng(32, 0).uniform(-1, 1, len(pts)).astype(np.float32)
    g[::17] = 0.0
    got = _adjoint(itp, torch.from_numpy(pts).cuda(), torch.from_numpy(g).cuda(), 1).cpu().numpy()
    shape = (len(lat.cosets),) + dims
    o = OracleSpline(name)
    ref = o.adjoint(lat.D, lat.cosets, shape, pts, g)
    bound = o.adjoint(lat.D, lat.cosets, shape, pts, np.abs(g))
    err = np.abs(got - ref)
    assert np.all(err <= 4e-6 * bound + 1e-7), (err.max(), bound.max())


@pytest.mark.parametrize("name,dims,n", [("bcc_quintic", (40, 36, 44), 300_001), ("fcc_6dir", (33, 40, 29), 200_003),
                                         ("cc_7dir", (50, 47, 52), 200_001)])
def test_binned_adjoint_equals_scatter(name, dims, n):
    # volumes spanning many bins with ragged edges, against the unbinned scatter
    torch = require_cuda()
    itp = make_interpolator(name, dims)
    lo, hi = interior_box(name, dims)
    pts = torch.from_numpy(uniform_points(make_rng(33, 0), n, lo - 3, hi + 3)).cuda()
    g = torch.from_numpy(make_rng(34, 0).uniform(-1, 1, n).astype(np.float32)).cuda()
    a = _adjoint(itp, pts, g, 1)
    b = _adjoint(itp, pts, g, 0)
    bound = _adjoint(itp, pts, g.abs(), 0)
    assert float(bound.max()) > 0
    assert bool(torch.all((a - b).abs() <= 8e-6 * bound + 2e-7)), float((a - b).abs().max())


def test_binned_adjoint_clustered_queries():
    # 200,000 queries inside two cells: one bin holds them all and is split into several work
    # items (chunks of 32768 queries), each adding its own box
    torch = require_cuda()
    name, dims = "bcc_quintic", (24, 24, 24)
    itp = make_interpolator(name, dims)
    rng = make_rng(35, 0)
    pts = (20.0 + rng.uniform(0, 3.5, (200_000, 3))).astype(np.float32)
    g = rng.uniform(-1, 1, 200_000).astype(np.float32)
    pt, gt = torch.from_numpy(pts).cuda(), torch.from_numpy(g).cuda()
    a = _adjoint(itp, pt, gt, 1)
    b = _adjoint(itp, pt, gt, 0)
    bound = _adjoint(itp, pt, gt.abs(), 0)
    assert bool(torch.all((a - b).abs() <= 8e-6 * bound + 2e-7)), float((a - b).abs().max())


def test_binned_adjoint_full_size_sampled():
    # the bench workload (BCC quintic, 2 x 128^3, 2^24 random queries, default options: the
    # binned path) on sampled coefficients: the oracle sums the contributions of every query in a
    # small box around each sampled site
    torch = require_cuda()
    wl = WORKLOADS["bcc_quintic_128"]
    sp, lat, xi, detl = spline_setup(wl.spline)
    itp = make_interpolator(wl.spline, wl.dims)
    lo, hi = interior_box(wl.spline, wl.dims)
    n = 1 << 24
    pts_h = uniform_points(make_rng(wl.seed, 0), n, lo, hi)
    g_h = make_rng(wl.seed, 5).uniform(-1, 1, n).astype(np.float32)
    dc = torch.zeros(itp.shape, device="cuda")
    itp.set_option("adjoint_bins", -1)
    itp.backward(torch.from_numpy(pts_h).cuda(), torch.from_numpy(g_h).cuda(), dc)
    got = dc.cpu().numpy()
    o = OracleSpline(wl.spline)
    rng = make_rng(36, 0)
    D = lat.D
    hw = np.asarray(o.halfwidth)
    for _ in range(24):
        k = int(rng.integers(0, len(lat.cosets)))
        i = rng.integers(2, np.asarray(wl.dims) - 2)
        site = D * i + np.asarray(lat.cosets[k])
        near = np.all(np.abs(pts_h - site) < hw + 1e-3, axis=1)
        z = pts_h[near].astype(np.float64) - site
        ref = float((o.phi(z) * g_h[near]).sum())
        bound = float((o.phi(z) * np.abs(g_h[near])).sum())
        assert abs(got[(k,) + tuple(i)] - ref) <= 4e-6 * bound + 1e-7, (k, i, got[(k,) + tuple(i)], ref)
