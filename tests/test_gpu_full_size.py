"""Full-size parity for the workloads other than the headline one, in the launch configuration of
bench.py (the default call path of each workload); outputs sampled and checked against the FP64
oracle, at the tolerances of the parity tests.

* BCC linear, 2 x 16^3 FP64 coefficients uniform in [-1, 1], all 10^4 interior queries (value);
* FCC 6-direction, 4 x 128^3 signal samples, 2^22 queries: value, gradient and the adjoint;
* FCC 6-direction fit: 200 Adam steps on 4 x 128^3 coefficients from 2^22 samples of the
  Marschner-Lobb signal through the hand-written adjoint, with the loss gradient checked against
  the oracle's adjoint and central differences at that size;
* D4*, 2 x 48^4 coefficients uniform in [-1, 1], 2^24 queries (value);
* the 64-volume batch (edges log-uniform in 32..256, four splines, 2^20 queries each) plus the
  D4* volume, one graph-replayed batched launch;
* the largest BCC quintic volume the 32-bit element offsets allow (2 x 1014^3), queries at both
  corners.
"""
import numpy as np
import pytest

import oracle
from synth import (LATTICES, SPLINES, WORKLOADS, batch_volumes, coefficients, hashed_coefficients, interior_box, make_rng,
                   marschner_lobb, uniform_points)

from _gpu_common import VALUE_TOL, OracleSpline, grad_bound, make_interpolator, require_cuda, spline_setup

pytestmark = pytest.mark.gpu


def test_bcc_linear_16_fp64_coefficients_all_queries():
    torch = require_cuda()
    wl = WORKLOADS["bcc_linear_16"]
    sp, lat, xi, detl = spline_setup(wl.spline)
    itp = make_interpolator(wl.spline, wl.dims)
    c = coefficients(wl, np.float64)
    itp.set_coeffs(torch.from_numpy(c).cuda())                # FP64 source, rounded once to FP32
    lo, hi = interior_box(wl.spline, wl.dims)
    pts = uniform_points(make_rng(wl.seed, 0), wl.queries, lo, hi)
    got = itp.eval(torch.from_numpy(pts).cuda()).cpu().numpy()
    ref = oracle.eval_sum(oracle.Spline(xi, detl), lat.D, lat.cosets, c, pts.astype(np.float64))
    assert len(pts) == 10_000
    assert np.abs(got - ref).max() <= VALUE_TOL * np.abs(c).max()


def _sampled_adjoint_check(o, lat, dims, pts_h, g_h, got, rng, nsites=16, atol=1e-7):
    hw = np.asarray(o.halfwidth)
    for _ in range(nsites):
        k = int(rng.integers(0, len(lat.cosets)))
        i = rng.integers(2, np.asarray(dims) - 2)
        site = lat.D * i + np.asarray(lat.cosets[k])
        near = np.all(np.abs(pts_h - site) < hw + 1e-3, axis=1)
        z = pts_h[near].astype(np.float64) - site
        ref = float((o.phi(z) * g_h[near]).sum())
        bound = float((o.phi(z) * np.abs(g_h[near])).sum())
        assert bound > 0
        assert abs(got[(k,) + tuple(i)] - ref) <= 4e-6 * bound + atol, (k, i, got[(k,) + tuple(i)], ref)


def test_fcc_6dir_128_value_gradient_adjoint_sampled():
    torch = require_cuda()
    wl = WORKLOADS["fcc_6dir_128"]
    sp, lat, xi, detl = spline_setup(wl.spline)
    itp = make_interpolator(wl.spline, wl.dims)
    c = coefficients(wl)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    lo, hi = interior_box(wl.spline, wl.dims)
    pts_h = uniform_points(make_rng(wl.seed, 0), wl.queries, lo, hi)
    pts = torch.from_numpy(pts_h).cuda()
    val, grad = itp.eval_grad(pts)
    v0 = itp.eval(pts)
    idx = make_rng(wl.seed, 98).choice(wl.queries, 512, replace=False)
    o = OracleSpline(wl.spline)
    ref_v, ref_g = o.eval_sum(lat.D, lat.cosets, c, pts_h[idx], grad=True)
    cmax = np.abs(c).max()
    G = grad_bound(wl.spline, pts_h[idx[:32]])
    assert np.abs(v0.cpu().numpy()[idx] - ref_v).max() <= VALUE_TOL * cmax
    assert np.abs(val.cpu().numpy()[idx] - ref_v).max() <= VALUE_TOL * cmax
    assert np.abs(grad.cpu().numpy()[idx] - ref_g).max() <= VALUE_TOL * cmax * G
    g_h = make_rng(wl.seed, 5).uniform(-1, 1, wl.queries).astype(np.float32)
    dc, _ = itp.backward(pts, torch.from_numpy(g_h).cuda())
    _sampled_adjoint_check(o, lat, wl.dims, pts_h, g_h, dc.cpu().numpy(), make_rng(wl.seed, 97))


def test_fcc_6dir_128_fit_200_adam_steps():
    """The fitting experiment at its configured size: 200 Adam steps (lr 0.05) from zero
    coefficients on 4 x 128^3 sites, 2^22 random samples of the Marschner-Lobb signal."""
    torch = require_cuda()
    from paper_2102_08514_b300.binding import lattice_interp
    from paper_2102_08514_b300.fit import fit, mse_loss
    wl = WORKLOADS["fcc_6dir_128"]
    sp, lat, xi, detl = spline_setup(wl.spline)
    itp = make_interpolator(wl.spline, wl.dims)
    lo, hi = interior_box(wl.spline, wl.dims)
    n = 1 << 22
    pts_h = uniform_points(make_rng(wl.seed, 11), n, lo, hi)
    phys = -1.0 + pts_h.astype(np.float64) / (lat.D * np.asarray(wl.dims) / 2.0)
    y_h = marschner_lobb(phys).astype(np.float32)
    pts, y = torch.from_numpy(pts_h).cuda(), torch.from_numpy(y_h).cuda()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record()
    c, losses = fit(itp, pts, y, steps=200, lr=0.05)
    end.record()
    torch.cuda.synchronize()
    print(f"fit: 200 steps in {start.elapsed_time(end):.1f} ms, loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    assert len(losses) == 200 and np.all(np.isfinite(losses))
    assert losses[-1] < 0.01 * losses[0]
    assert all(b <= a * 1.5 for a, b in zip(losses[::20], losses[20::20]))      # no blow-up along the way
    # the loss gradient at the fitted coefficients: adjoint vs the oracle's closed form on sampled
    # coefficients, and vs central differences of the FP64 loss
    cg = c.clone().requires_grad_(True)
    f = lattice_interp(pts, cg, itp)
    mse_loss(f, y).backward()
    g = cg.grad.cpu().numpy()
    r = ((2.0 / n) * (f.detach().double() - y.double())).cpu().numpy()
    o = OracleSpline(wl.spline)
    _sampled_adjoint_check(o, lat, wl.dims, pts_h, r, g, make_rng(wl.seed, 12), nsites=8, atol=1e-14)
    flat = np.argsort(-np.abs(g).ravel())[:3]
    h = 1e-2
    for idx in flat:
        k = np.unravel_index(idx, itp.shape)
        cp, cm = c.clone(), c.clone()
        cp[k] += h
        cm[k] -= h
        with torch.no_grad():
            lp = float(mse_loss(lattice_interp(pts, cp, itp), y))
            lm = float(mse_loss(lattice_interp(pts, cm, itp), y))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 2e-3 * abs(g[k]) + 1e-9, (k, fd, g[k])


def test_d4s_8dir_48_value_sampled():
    torch = require_cuda()
    wl = WORKLOADS["d4s_8dir_48"]
    sp, lat, xi, detl = spline_setup(wl.spline)
    itp = make_interpolator(wl.spline, wl.dims)
    c = coefficients(wl)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    lo, hi = interior_box(wl.spline, wl.dims)
    pts_h = uniform_points(make_rng(wl.seed, 0), wl.queries, lo, hi)
    got = itp.eval(torch.from_numpy(pts_h).cuda()).cpu().numpy()
    idx = make_rng(wl.seed, 96).choice(wl.queries, 160, replace=False)
    ref = OracleSpline(wl.spline).eval_sum(lat.D, lat.cosets, c, pts_h[idx])
    assert np.abs(got[idx] - ref).max() <= VALUE_TOL * np.abs(c).max()


def test_batch64_and_d4s_full_size_sampled():
    torch = require_cuda()
    from paper_2102_08514_b300.binding import Batch, Interpolator
    vols = batch_volumes(64) + [("d4s_8dir", (48, 48, 48, 48))]
    items, data = [], []
    for v, (name, dims) in enumerate(vols):
        sp = SPLINES[name]
        lat = LATTICES[sp.lattice]
        itp = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), dims, "f32")
        rng = make_rng(2106, v)
        c = rng.uniform(-1, 1, itp.shape).astype(np.float32)
        itp.set_coeffs(torch.from_numpy(c).cuda())
        nq = (1 << 24) if name == "d4s_8dir" else (1 << 20)
        lo, hi = interior_box(name, dims)
        pts_h = uniform_points(rng, nq, lo, hi)
        out = torch.full((nq,), float("nan"), device="cuda")
        items.append((itp, torch.from_numpy(pts_h).cuda(), out))
        data.append((name, lat, c, pts_h))
    assert all(32 <= d <= 256 for name, dims in vols[:64] for d in dims)
    batch = Batch(items)
    batch.autotune()
    for _, _, out in items:
        out.fill_(float("nan"))
    batch.run()
    torch.cuda.synchronize()
    for v, ((itp, dp, out), (name, lat, c, pts_h)) in enumerate(zip(items, data)):
        assert not bool(torch.isnan(out).any()), name
        idx = make_rng(95, v).choice(len(pts_h), 24 if name != "d4s_8dir" else 64, replace=False)
        ref = OracleSpline(name).eval_sum(lat.D, lat.cosets, c, pts_h[idx])
        got = out.cpu().numpy()[idx]
        assert np.abs(got - ref).max() <= VALUE_TOL * np.abs(c).max(), (v, name)


def test_bcc_quintic_largest_volume_both_corners():
    """Maximum size: the largest cube of BCC quintic coefficients whose padded FP32 arrays fit the
    library's 32-bit element offsets (2 x 1014^3 sites, 8.3 GB; 1015 is refused with ESIZE before
    any allocation, test_abi), hashed coefficients generated on the device slab by slab.  Queries
    near both corners and inside, value and gradient, each against the oracle on the block of
    coefficients around it (shifted by a lattice vector; zero outside the volume)."""
    torch = require_cuda()
    name, n = "bcc_quintic", 1014
    sp, lat, xi, detl = spline_setup(name)
    dims = (n, n, n)
    itp = make_interpolator(name, dims)
    M = len(lat.cosets)
    c = torch.empty((M,) + dims, device="cuda")
    J = torch.arange(n, device="cuda", dtype=torch.int64)
    for k in range(M):
        for i0 in range(0, n, 64):
            I = torch.arange(i0, min(n, i0 + 64), device="cuda", dtype=torch.int64)
            c[k, i0:i0 + len(I)] = hashed_coefficients(k, (I[:, None, None], J[None, :, None], J[None, None, :]), xp=torch)
    itp.set_coeffs(c)
    del c
    lo, hi = interior_box(name, dims)
    rng = make_rng(3007, 0)
    pts = np.concatenate([uniform_points(rng, 32, lo, lo + 4.0), uniform_points(rng, 32, hi - 4.0, hi),
                          uniform_points(rng, 32, lo, hi)])
    val, grad = itp.eval_grad(torch.from_numpy(pts).cuda())
    val, grad = val.cpu().numpy(), grad.cpu().numpy()
    o = oracle.Spline(xi, detl)
    G = grad_bound(name, pts)
    B = 10
    for q, x in enumerate(pts.astype(np.float64)):
        i0 = np.floor(x / lat.D).astype(np.int64) - 4
        idx = [np.arange(i0[a], i0[a] + B) for a in range(3)]
        blk = np.stack([hashed_coefficients(k, (idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]))
                        for k in range(M)]).astype(np.float64)
        inside = [(v >= 0) & (v < n) for v in idx]
        blk *= (inside[0][:, None, None] & inside[1][None, :, None] & inside[2][None, None, :])[None]
        ref_v, ref_g = oracle.eval_sum(o, lat.D, lat.cosets, blk, (x - lat.D * i0)[None], grad=True)
        assert abs(val[q] - ref_v[0]) <= VALUE_TOL, (q, x, val[q], ref_v[0])
        assert np.abs(grad[q] - ref_g[0]).max() <= VALUE_TOL * G, (q, x, grad[q], ref_g[0])
