"""Ray mode (orthographic rays through the interior box, per-pixel sums of f and grad f) against
the oracle evaluated at the GPU's own sample points."""
import numpy as np
import pytest

import oracle
from synth import LATTICES, SPLINES, make_rng, ray_points, ray_setup

from _gpu_common import VALUE_TOL, OracleSpline, grad_bound, make_interpolator, require_cuda

pytestmark = pytest.mark.gpu


def _geometry(setup, W, H, steps):
    eu, ev = setup["eu"], setup["ev"]
    origin = setup["centre"] - setup["half_u"] * eu - setup["half_v"] * ev
    du = (2.0 * setup["half_u"] / W) * eu
    dv = (2.0 * setup["half_v"] / H) * ev
    return origin, du, dv


@pytest.mark.parametrize("name,grad", [("bcc_quintic", True), ("bcc_quintic", False), ("cc_7dir", True),
                                       ("bcc_voronoi2", True), ("fcc_voronoi1", False)])
def test_rays_match_oracle(name, grad):
    torch = require_cuda()
    from paper_2102_08514_b300.binding import interp_eval_rays, make_rays
    sp = SPLINES[name]
    lat = LATTICES[sp.lattice]
    dims = (14, 14, 14)
    itp = make_interpolator(name, dims)
    c = make_rng(61, 1).uniform(-1, 1, itp.shape).astype(np.float32)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    W, H, steps = 37, 21, 48                 # ragged against the 16 x 8 pixel blocks
    setup = ray_setup(name, dims, W, H, steps)
    origin, du, dv = _geometry(setup, W, H, steps)
    rays = make_rays(origin, du, dv, setup["d"], setup["lo"], setup["hi"], W, H, steps)
    out = torch.empty(W * H * (4 if grad else 1), device="cuda")
    pts = torch.empty(W * H * steps * 3, device="cuda")
    interp_eval_rays(itp.handle, rays, out, with_grad=grad, pts_out=pts)
    out = out.cpu().numpy().reshape(H, W, -1)
    pts = pts.cpu().numpy().reshape(H, W, steps, 3)
    # the sample points follow the host-side definition (FP32 rounding aside)
    pix = np.array([[px, py] for py in range(H) for px in range(W)])
    ref_pts, valid = ray_points(setup, pix)
    got_valid = ~np.isnan(pts.reshape(-1, steps, 3)[:, 0, 0])
    assert np.array_equal(got_valid, valid)
    assert np.abs(pts.reshape(-1, steps, 3)[valid] - ref_pts[valid]).max() < 1e-3
    assert np.all(out.reshape(H * W, -1)[~valid] == 0.0)
    # sums against the oracle at the GPU's points, for a sample of pixels
    o = OracleSpline(name)
    sel = make_rng(62, 0).choice(np.flatnonzero(valid), 8 if sp.order > 1 else 24, replace=False)
    P = pts.reshape(-1, steps, 3)[sel].reshape(-1, 3).astype(np.float64)
    if grad:
        v, g = o.eval_sum(lat.D, lat.cosets, c, P, grad=True)
        G = grad_bound(name, P[::97])
        ref = np.concatenate([v.reshape(-1, steps).sum(1)[:, None], g.reshape(-1, steps, 3).sum(1)], axis=1)
        got = out.reshape(H * W, 4)[sel]
        cm = np.abs(c).max()
        assert np.abs(got[:, 0] - ref[:, 0]).max() <= steps * VALUE_TOL * cm
        assert np.abs(got[:, 1:] - ref[:, 1:]).max() <= steps * VALUE_TOL * cm * G
    else:
        v = o.eval_sum(lat.D, lat.cosets, c, P)
        ref = v.reshape(-1, steps).sum(1)
        got = out.reshape(H * W)[sel]
        assert np.abs(got - ref).max() <= steps * VALUE_TOL * np.abs(c).max()


@pytest.mark.parametrize("name,steps", [("bcc_voronoi1", 48), ("fcc_voronoi2", 48), ("bcc_voronoi2", 700)])
def test_binned_rays_equal_plain_rays(name, steps):
    # multi-piece splines march rays with the piece-binned kernel (whole rays per tile, sums in
    # step and coset order); the handle option "binned" = 0 selects the plain kernel: identical sums
    torch = require_cuda()
    from paper_2102_08514_b300.binding import interp_eval_rays, make_rays
    dims = (12, 13, 11)
    itp = make_interpolator(name, dims)
    itp.set_coeffs(torch.from_numpy(make_rng(63, 1).uniform(-1, 1, itp.shape).astype(np.float32)).cuda())
    W, H = 29, 17
    setup = ray_setup(name, dims, W, H, steps)
    origin, du, dv = _geometry(setup, W, H, steps)
    rays = make_rays(origin, du, dv, setup["d"], setup["lo"], setup["hi"], W, H, steps)
    res = []
    for flag in ("1", "0"):
        itp.set_option("binned", int(flag))
        for grad in (False, True):
            out = torch.full((W * H * (4 if grad else 1),), 7.0, device="cuda")
            pts = torch.empty(W * H * steps * 3, device="cuda")
            interp_eval_rays(itp.handle, rays, out, with_grad=grad, pts_out=pts)
            res.append((out, pts))
    for (a, pa), (b, pb) in zip(res[:2], res[2:]):
        assert torch.equal(a, b)
        assert torch.equal(torch.nan_to_num(pa, nan=7.0), torch.nan_to_num(pb, nan=7.0))


def test_rays_reject_4d_and_half_storage():
    torch = require_cuda()
    from paper_2102_08514_b300.binding import (INTERP_EUNSUPPORTED, InterpError, Interpolator, interp_eval_rays,
                                               make_rays)
    lat = LATTICES["bcc"]
    itp = Interpolator(np.asarray(lat.L), np.asarray(SPLINES["bcc_quintic"].xi), (8, 8, 8), "f16")
    rays = make_rays([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [9, 9, 9], 4, 4, 8)
    out = torch.empty(16, device="cuda")
    with pytest.raises(InterpError) as e:
        interp_eval_rays(itp.handle, rays, out)
    assert e.value.status == INTERP_EUNSUPPORTED
