"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle, element by element.

Tolerances (the benchmark spec): cell indices bit-exact; piece indices exact or within 1e-6 of a piece
boundary; values max-abs <= 2e-6 * max|c|; gradients <= 2e-6 * max|c| * G with
G = max_x sum_n |grad phi(x - n)|_inf estimated by the oracle; adjoint per coefficient <= 4e-6 *
sum_q |g_q| phi(x_q - n) + 1e-7 (FP32 atomics in arbitrary order).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from synth import LATTICES, SPLINES, WORKLOADS, coefficients, interior_box, make_rng, uniform_points

from _gpu_common import (VALUE_TOL, OracleSpline, grad_bound, make_interpolator, mixed_points, require_cuda,
                         spline_setup, tables)

pytestmark = pytest.mark.gpu

SPLINES_ALL = ["bcc_linear", "bcc_quintic", "fcc_6dir", "cc_7dir", "d4s_8dir", "d4_8dir", "bcc_quartic", "cc_linear_rd",
               "cc_voronoi1", "cc_voronoi2", "cc_voronoi3", "bcc_voronoi1", "bcc_voronoi2", "fcc_voronoi1",
               "fcc_voronoi2"]
# small cases the oracle finishes in seconds, spanning several thread blocks and a ragged tail
SMALL = {"bcc_linear": (12, 4133), "bcc_quintic": (12, 2085), "fcc_6dir": (10, 3011), "cc_7dir": (14, 2107),
         "d4s_8dir": (7, 1093), "d4_8dir": (6, 517), "bcc_quartic": (12, 2091), "cc_linear_rd": (14, 3003), "cc_voronoi1": (14, 4099),
         "cc_voronoi2": (14, 2049), "cc_voronoi3": (12, 389), "bcc_voronoi1": (12, 4111),
         "bcc_voronoi2": (10, 397), "fcc_voronoi1": (10, 3079), "fcc_voronoi2": (10, 1031)}


def _interp(name, dims, storage="f32"):
    torch = require_cuda()
    return torch, make_interpolator(name, dims, storage)


def _coeffs(name, dims, seed):
    lat = LATTICES[SPLINES[name].lattice]
    rng = make_rng(seed, 3)
    return rng.uniform(-1, 1, (len(lat.cosets),) + tuple(dims)).astype(np.float32)


@pytest.mark.parametrize("name", SPLINES_ALL)
def test_value_parity_small(name):
    n_axis, nq = SMALL[name]
    sp, lat, xi, detl = spline_setup(name)
    dims = (n_axis,) * xi.shape[0]
    torch, itp = _interp(name, dims)
    c = _coeffs(name, dims, 1)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    pts = mixed_points(name, dims, nq, 2)
    got = itp.eval(torch.from_numpy(pts).cuda()).cpu().numpy()
    ref = OracleSpline(name).eval_sum(lat.D, lat.cosets, c, pts)
    err = np.abs(got - ref)
    assert err.max() <= VALUE_TOL * np.abs(c).max(), (err.max(), int(err.argmax()))


@pytest.mark.parametrize("name", SPLINES_ALL)
def test_cell_and_piece_indices(name):
    n_axis, nq = SMALL[name]
    sp, lat, xi, detl = spline_setup(name)
    s = xi.shape[0]
    dims = (n_axis,) * s
    torch, itp = _interp(name, dims)
    pts = mixed_points(name, dims, nq, 3)
    cells, piece = itp.debug_indices(torch.from_numpy(pts).cuda())
    cells = cells.cpu().numpy()
    piece = piece.cpu().numpy()
    ref_cells, offs = oracle.cells(s, lat.D, lat.cosets, pts.astype(np.float64))
    assert np.array_equal(cells, ref_cells)
    # the GPU's piece label j must name a polytope containing the oracle's folded offset
    tab = tables()[name]
    yf = oracle.folded_offsets(offs)
    polys = []
    for pc in tab["pieces"]:
        A = np.array([[float(Fraction(a)) for a in row[0]] for row in pc["ineqs"]])
        b = np.array([float(Fraction(row[1])) for row in pc["ineqs"]])
        polys.append((A / np.linalg.norm(A, axis=1, keepdims=True), b / np.linalg.norm(A, axis=1)))
    bad = 0
    for q in range(len(pts)):
        for k in range(len(lat.cosets)):
            A, b = polys[piece[q, k]]
            viol = (A @ yf[q, k] - b).max()
            bad += viol > 1e-6
    assert bad == 0


@pytest.mark.parametrize("name", SPLINES_ALL)
def test_gradient_parity(name):
    n_axis, nq = SMALL[name]
    sp, lat, xi, detl = spline_setup(name)
    s = xi.shape[0]
    dims = (n_axis,) * s
    torch, itp = _interp(name, dims)
    c = _coeffs(name, dims, 4)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    lo, hi = interior_box(name, dims)
    pts = uniform_points(make_rng(5, 0), nq // 2, lo, hi)
    val, grad = itp.eval_grad(torch.from_numpy(pts).cuda())
    ref_v, ref_g = OracleSpline(name).eval_sum(lat.D, lat.cosets, c, pts, grad=True)
    G = grad_bound(name, pts[:32])
    cmax = np.abs(c).max()
    assert np.abs(val.cpu().numpy() - ref_v).max() <= VALUE_TOL * cmax
    gerr = np.abs(grad.cpu().numpy() - ref_g).max()
    assert gerr <= VALUE_TOL * cmax * G, (gerr, G)


@pytest.mark.parametrize("name", SPLINES_ALL)
def test_adjoint_parity(name):
    n_axis, nq = SMALL[name]
    sp, lat, xi, detl = spline_setup(name)
    s = xi.shape[0]
    dims = (n_axis,) * s
    torch, itp = _interp(name, dims)
    pts = mixed_points(name, dims, nq, 6)
    g = make_rng(7, 0).uniform(-1, 1, len(pts)).astype(np.float32)
    shape = (len(lat.cosets),) + dims
    dpre = make_rng(8, 0).uniform(-1, 1, shape).astype(np.float32)      # accumulated into (+=)
    dc = torch.from_numpy(dpre.copy()).cuda()
    itp.backward(torch.from_numpy(pts).cuda(), torch.from_numpy(g).cuda(), dc)
    sp_o = OracleSpline(name)
    ref = sp_o.adjoint(lat.D, lat.cosets, shape, pts, g)
    bound = sp_o.adjoint(lat.D, lat.cosets, shape, pts, np.abs(g))
    err = np.abs(dc.cpu().numpy() - dpre - ref)
    assert np.all(err <= 4e-6 * bound + 1e-7), (err.max(), bound.max())


@pytest.mark.parametrize("name", ["bcc_linear", "cc_linear_rd", "cc_voronoi1", "bcc_voronoi1", "fcc_voronoi1"])
def test_gradient_at_exact_ties(name):
    # continuous, not C^1 splines: at points exactly on mesh planes (integer, half and quarter
    # coordinates, and sums of them) the gradient is the one-sided limit along the fixed world
    # direction v = (1, 2^-12, 2^-24), on the GPU (every coset and fold decision) as in the oracle
    n_axis = SMALL[name][0]
    sp, lat, xi, detl = spline_setup(name)
    dims = (n_axis,) * 3
    torch, itp = _interp(name, dims)
    c = _coeffs(name, dims, 24)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    lo, hi = interior_box(name, dims)
    rng = make_rng(25, 0)
    pts = (np.round(rng.uniform(lo, hi, (1500, 3)) * 4) / 4).astype(np.float32)
    pts[::3, 1] = (np.round(rng.uniform(lo[1], hi[1], 500) * 2 ** 12) / 2 ** 12).astype(np.float32)
    pts[1::3, 0] = (np.floor(pts[1::3, 1]) + 0.5 - (pts[1::3, 1] - np.floor(pts[1::3, 1]))).astype(np.float32)
    for flag in ("1", "0") if SPLINES[name].order else ("0",):
        itp.set_option("binned", int(flag))         # binned and plain kernels alike
        val, grad = itp.eval_grad(torch.from_numpy(pts).cuda())
        ref_v, ref_g = OracleSpline(name).eval_sum(lat.D, lat.cosets, c, pts, grad=True)
        cmax = np.abs(c).max()
        G = grad_bound(name, pts[:16])
        assert np.abs(val.cpu().numpy() - ref_v).max() <= VALUE_TOL * cmax
        gerr = np.abs(grad.cpu().numpy() - ref_g).max()
        assert gerr <= VALUE_TOL * cmax * G, (gerr, int(np.abs(grad.cpu().numpy() - ref_g).max(axis=1).argmax()))


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc_6dir"])
def test_pullback_dpts(name):
    n_axis, nq = SMALL[name]
    sp, lat, xi, detl = spline_setup(name)
    dims = (n_axis,) * xi.shape[0]
    torch, itp = _interp(name, dims)
    c = _coeffs(name, dims, 9)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    lo, hi = interior_box(name, dims)
    pts = torch.from_numpy(uniform_points(make_rng(10, 0), 1000, lo, hi)).cuda()
    g = torch.linspace(-1, 1, 1000, device="cuda")
    _, grad = itp.eval_grad(pts)
    dpts = torch.empty_like(grad)
    from paper_2102_08514_b300.binding import interp_backward
    interp_backward(itp.handle, pts, g, None, dpts)      # dcoeffs = NULL: dpts only
    assert torch.allclose(dpts, g[:, None] * grad, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("name", ["bcc_quintic", "cc_7dir", "fcc_6dir"])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_reduced_precision_storage(name, storage):
    # stated accuracy: against the oracle on the dequantised coefficients the FP32 arithmetic
    # bound holds; against the original coefficients the quantisation error dominates
    n_axis, nq = SMALL[name]
    sp, lat, xi, detl = spline_setup(name)
    dims = (n_axis,) * xi.shape[0]
    torch, itp = _interp(name, dims, storage)
    c = _coeffs(name, dims, 11)
    tdt = torch.float16 if storage == "f16" else torch.bfloat16
    cq = torch.from_numpy(c).to(tdt)
    itp.set_coeffs(cq.cuda())
    lo, hi = interior_box(name, dims)
    pts = uniform_points(make_rng(12, 0), nq // 2, lo, hi)
    got = itp.eval(torch.from_numpy(pts).cuda()).cpu().numpy()
    sp_o = oracle.Spline(xi, detl)
    ref_q = oracle.eval_sum(sp_o, lat.D, lat.cosets, cq.double().numpy(), pts.astype(np.float64))
    ref = oracle.eval_sum(sp_o, lat.D, lat.cosets, c.astype(np.float64), pts.astype(np.float64))
    assert np.abs(got - ref_q).max() <= VALUE_TOL * np.abs(c).max()
    unit = 2.0 ** -11 if storage == "f16" else 2.0 ** -8
    assert np.abs(got - ref).max() <= 2 * unit * np.abs(c).max()


def test_edge_cases():
    torch = require_cuda()
    name = "bcc_quintic"
    dims = (8, 8, 8)
    _, itp = _interp(name, dims)
    c = _coeffs(name, dims, 13)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    # empty input
    out = torch.empty(0, device="cuda")
    from paper_2102_08514_b300.binding import interp_eval
    interp_eval(itp.handle, torch.empty(0, 3, device="cuda"), out)
    # NaN / inf propagate; far away is exactly zero
    p = torch.tensor([[float("nan"), 3.0, 3.0], [3.0, float("inf"), 3.0], [1e6, 1e6, 1e6], [-1e30, 0.0, 0.0]],
                     device="cuda")
    v = itp.eval(p).cpu().numpy()
    assert np.isnan(v[0]) and np.isnan(v[1]) and v[2] == 0.0 and v[3] == 0.0
    # host coefficients (F64 source) equal device F32 source after rounding
    itp2 = _interp(name, dims)[1]
    itp2.set_coeffs(torch.from_numpy(c.astype(np.float64)))
    lo, hi = interior_box(name, dims)
    q = torch.from_numpy(uniform_points(make_rng(14, 0), 777, lo, hi)).cuda()
    assert torch.equal(itp.eval(q), itp2.eval(q))


def test_create_rejects_bad_input():
    require_cuda()
    from paper_2102_08514_b300.binding import InterpError, interp_create, INTERP_EUNSUPPORTED, INTERP_EINVAL
    sp, lat, xi, detl = spline_setup("bcc_quintic")
    with pytest.raises(InterpError) as e:
        interp_create(np.asarray(lat.L), xi[:, :5], (8, 8, 8))
    assert e.value.status == INTERP_EUNSUPPORTED
    with pytest.raises(InterpError) as e:
        interp_create(np.zeros((3, 3)), xi, (8, 8, 8))
    assert e.value.status == INTERP_EINVAL
    # column order and signs do not matter
    perm = np.random.default_rng(0).permutation(xi.shape[1])
    h = interp_create(np.asarray(lat.L), -xi[:, perm], (8, 8, 8))
    from paper_2102_08514_b300.binding import interp_destroy
    interp_destroy(h)


def test_full_size_headline_workload_sampled():
    """BCC quintic on 2 x 128^3 FP32 signal samples with 2^24 queries, in the bench's launch
    configuration; sampled outputs against the oracle."""
    torch = require_cuda()
    wl = WORKLOADS["bcc_quintic_128"]
    sp, lat, xi, detl = spline_setup(wl.spline)
    _, itp = _interp(wl.spline, wl.dims)
    c = coefficients(wl)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    lo, hi = interior_box(wl.spline, wl.dims)
    pts = uniform_points(make_rng(wl.seed, 0), wl.queries, lo, hi)
    dp = torch.from_numpy(pts).cuda()
    val, grad = itp.eval_grad(dp)
    v0 = itp.eval(dp)
    idx = make_rng(wl.seed, 99).choice(wl.queries, 512, replace=False)
    sp_o = oracle.Spline(xi, detl)
    ref_v, ref_g = oracle.eval_sum(sp_o, lat.D, lat.cosets, c.astype(np.float64), pts[idx].astype(np.float64),
                                   grad=True)
    cmax = np.abs(c).max()
    G = grad_bound(wl.spline, pts[idx[:32]])
    assert np.abs(v0.cpu().numpy()[idx] - ref_v).max() <= VALUE_TOL * cmax
    assert np.abs(val.cpu().numpy()[idx] - ref_v).max() <= VALUE_TOL * cmax
    assert np.abs(grad.cpu().numpy()[idx] - ref_g).max() <= VALUE_TOL * cmax * G


@pytest.mark.parametrize("name", ["fcc_6dir", "d4s_8dir", "d4_8dir", "bcc_voronoi1", "fcc_voronoi1", "fcc_voronoi2",
                                  "bcc_voronoi2"])
def test_piece_binned_kernel_equals_plain_kernel(name):
    # multi-piece splines with much divergent work run a piece-binned kernel by default
    # (interp_info_t.binned); the handle option "binned" selects either: the plain kernel shares
    # the loads and the Horner evaluation between the pieces, but each piece's sums run in the
    # same order, so the results agree exactly
    n_axis, nq = SMALL[name]
    sp, lat, xi, detl = spline_setup(name)
    dims = (n_axis,) * xi.shape[0]
    torch, itp = _interp(name, dims)
    assert itp.info.binned == (name in ("d4s_8dir", "d4_8dir", "bcc_voronoi1", "fcc_voronoi2", "bcc_voronoi2"))
    itp.set_coeffs(torch.from_numpy(_coeffs(name, dims, 15)).cuda())
    pts = torch.from_numpy(mixed_points(name, dims, 5000, 16)).cuda()
    g = torch.linspace(-1, 1, pts.shape[0], device="cuda")
    from paper_2102_08514_b300.binding import interp_backward
    res = []
    for flag in ("1", "0"):
        itp.set_option("binned", int(flag))
        v = itp.eval(pts)
        v2, gr = itp.eval_grad(pts)
        dp = torch.empty_like(gr)
        interp_backward(itp.handle, pts, g, None, dp)
        res.append((v, v2, gr, dp))
    for a, b in zip(*res):
        assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))


@pytest.mark.parametrize("name", ["bcc_quintic", "bcc_quartic", "cc_voronoi2"])
def test_cooperative_gathers_equal_per_lane_gathers(name):
    # one-piece splines of 24 to 32 sites gather, for a warp of random queries, one query's
    # stencil per load instruction through a shared-memory table, and per lane when the warp's
    # queries lie within 8 cells per axis (here: the same queries spatially sorted); the sums run
    # in the same order either way, so values, gradients and pullbacks agree bit for bit
    sp, lat, xi, detl = spline_setup(name)
    dims = (24,) * xi.shape[0]
    torch, itp = _interp(name, dims)
    assert itp.info.coop == 1
    itp.set_coeffs(torch.from_numpy(_coeffs(name, dims, 41)).cuda())
    pts = torch.from_numpy(mixed_points(name, dims, 20011, 42)).cuda()
    perm, pts_s = itp.sort_points(pts)
    perm = perm.long()
    assert torch.equal(pts[perm], pts_s)
    g = torch.linspace(-1, 1, pts.shape[0], device="cuda")
    from paper_2102_08514_b300.binding import interp_backward
    res = []
    for p, gg in ((pts, g), (pts_s, g[perm])):
        v = itp.eval(p)
        v2, gr = itp.eval_grad(p)
        dp = torch.empty_like(gr)
        interp_backward(itp.handle, p, gg, None, dp)      # dcoeffs = NULL: the pullback only
        res.append((v, v2, gr, dp))
    for a, b in zip(res[0], res[1]):
        assert torch.equal(torch.nan_to_num(a[perm], nan=7.0), torch.nan_to_num(b, nan=7.0))
    assert _interp("cc_7dir", (8, 8, 8))[1].info.coop == 0 and _interp("fcc_6dir", (8, 8, 8))[1].info.coop == 0


def test_named_creation_matches_lattice_and_directions():
    # interp_create_named reaches the same tables as interp_create for a box spline; a Voronoi
    # spline's recorded generators never match a direction-matrix request
    torch = require_cuda()
    from paper_2102_08514_b300.binding import Interpolator, InterpError
    dims = (9, 10, 11)
    a = _interp("fcc_6dir", dims)[1]
    b = Interpolator.named("fcc_6dir", dims)
    c = _coeffs("fcc_6dir", dims, 21)
    a.set_coeffs(torch.from_numpy(c).cuda())
    b.set_coeffs(torch.from_numpy(c).cuda())
    pts = torch.from_numpy(mixed_points("fcc_6dir", dims, 3000, 22)).cuda()
    assert torch.equal(torch.nan_to_num(a.eval(pts), nan=7.0), torch.nan_to_num(b.eval(pts), nan=7.0))
    assert b.info.kind == 0 and Interpolator.named("bcc_voronoi2", dims).info.kind == 2
    sp, lat, xi, _ = spline_setup("fcc_voronoi1")          # FCC + its Voronoi generators x 2
    with pytest.raises(InterpError):
        Interpolator(np.asarray(lat.L), xi, dims)
    with pytest.raises(InterpError):
        Interpolator.named("no_such_spline", dims)


def test_eval_host_matches_device_path():
    # host buffers in, host buffers out, several chunks plus a ragged tail
    torch = require_cuda()
    from paper_2102_08514_b300.binding import interp_eval_host
    name = "bcc_quintic"
    dims = (20, 20, 20)
    _, itp = _interp(name, dims)
    itp.set_coeffs(torch.from_numpy(_coeffs(name, dims, 21)).cuda())
    lo, hi = interior_box(name, dims)
    n = (1 << 21) + 4321
    pts = torch.from_numpy(uniform_points(make_rng(22, 0), n, lo, hi)).pin_memory()
    out = torch.empty(n, pin_memory=True)
    grad = torch.empty(n, 3, pin_memory=True)
    interp_eval_host(itp.handle, pts, out, grad)
    torch.cuda.synchronize()
    v, g = itp.eval_grad(pts.cuda())
    assert torch.equal(out, v.cpu()) and torch.equal(grad, g.cpu())
    out2 = torch.empty(n, pin_memory=True)
    interp_eval_host(itp.handle, pts, out2)                          # value only
    torch.cuda.synchronize()
    assert torch.equal(out2, itp.eval(pts.cuda()).cpu())
