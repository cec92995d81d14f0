"""Fitting through the hand-written adjoint (FCC 6-direction): the autograd gradient against the
oracle's adjoint and against finite differences of the FP64 loss; Adam reduces the loss."""
import numpy as np
import pytest

import oracle
from synth import LATTICES, SPLINES, interior_box, make_rng, marschner_lobb, uniform_points

from _gpu_common import require_cuda

pytestmark = pytest.mark.gpu


def _problem(torch, dims=(12, 12, 12), n=20000):
    from paper_2102_08514_b300.binding import Interpolator
    sp = SPLINES["fcc_6dir"]
    lat = LATTICES["fcc"]
    itp = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), dims, "f32")
    lo, hi = interior_box("fcc_6dir", dims)
    pts = uniform_points(make_rng(71, 0), n, lo, hi)
    phys = -1.0 + pts.astype(np.float64) / (lat.D * np.asarray(dims) / 2.0)
    y = marschner_lobb(phys).astype(np.float32)
    return itp, lat, sp, torch.from_numpy(pts).cuda(), torch.from_numpy(y).cuda()


def test_loss_gradient_against_oracle_adjoint_and_fd():
    torch = require_cuda()
    from paper_2102_08514_b300.binding import lattice_interp
    from paper_2102_08514_b300.fit import mse_loss
    itp, lat, sp, pts, y = _problem(torch)
    c0 = torch.from_numpy(make_rng(72, 1).uniform(-1, 1, itp.shape).astype(np.float32)).cuda()
    c = c0.clone().requires_grad_(True)
    f = lattice_interp(pts, c, itp)
    loss = mse_loss(f, y)
    loss.backward()
    g = c.grad.cpu().numpy()
    # oracle: dloss/dc_n = (2/N) sum_q (f_q - y_q) phi(x_q - n), with the GPU's f
    N = pts.shape[0]
    r = (2.0 / N) * (f.detach().double() - y.double()).cpu().numpy()
    o = oracle.Spline(np.asarray(sp.xi), 2)
    ref = oracle.adjoint(o, lat.D, lat.cosets, itp.shape, pts.cpu().numpy().astype(np.float64), r)
    bound = oracle.adjoint(o, lat.D, lat.cosets, itp.shape, pts.cpu().numpy().astype(np.float64), np.abs(r))
    assert np.all(np.abs(g - ref) <= 4e-6 * bound + 1e-9)
    # central finite differences of the FP64 loss for a few coefficients
    flat = np.argsort(-np.abs(g).ravel())[:4]
    h = 1e-2
    for idx in flat:
        k = np.unravel_index(idx, itp.shape)
        cp, cm = c0.clone(), c0.clone()
        cp[k] += h
        cm[k] -= h
        with torch.no_grad():
            lp = float(mse_loss(lattice_interp(pts, cp, itp), y))
            lm = float(mse_loss(lattice_interp(pts, cm, itp), y))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-3 * abs(g[k]) + 1e-7, (fd, g[k])


def test_adam_fit_reduces_the_loss():
    torch = require_cuda()
    from paper_2102_08514_b300.fit import fit
    itp, lat, sp, pts, y = _problem(torch)
    c, losses = fit(itp, pts, y, steps=60, lr=0.05)
    assert losses[-1] < 0.05 * losses[0]
    assert np.all(np.isfinite(losses))
