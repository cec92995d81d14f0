"""GPU: the piece pre-sort.  For the splines where it measured faster (BCC V_2, the 8-coset D4)
calls of 2^16 or more queries sort the queries on the device by the pieces of their first cosets
(Sec. 4.3's sub-regions) before the piece-binned kernel, in chunks of 2^22, and return the
results to the callers' positions.  A query's sum does not depend on its tile's other queries, so
values, gradients and pullbacks equal the unsorted binned kernel's bit for bit; the adjoint's
atomic scatter agrees within rounding; under stream capture the call runs unsorted.
The handle option "presort" (0 / 1) forces the pre-sort off / on."""
import numpy as np
import pytest

from synth import LATTICES, SPLINES, interior_box, make_rng, uniform_points

from _gpu_common import VALUE_TOL, OracleSpline, grad_bound, make_interpolator, mixed_points, require_cuda

pytestmark = pytest.mark.gpu

# (grid sites per axis, queries): the BCC V_2 case spans two chunks of 2^22 plus a ragged tail
CASES = {"bcc_voronoi2": (12, (1 << 22) + 4999), "d4s_8dir": (8, 70001), "d4_8dir": (6, 65537),
         "fcc_voronoi2": (10, 9001), "bcc_voronoi1": (12, 9007)}


def _setup(name, n_axis, seed):
    torch = require_cuda()
    dims = (n_axis,) * len(SPLINES[name].xi)
    itp = make_interpolator(name, dims)
    lat = LATTICES[SPLINES[name].lattice]
    c = make_rng(seed, 3).uniform(-1, 1, (len(lat.cosets),) + dims).astype(np.float32)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    return torch, itp, dims, c


def _run_all(torch, itp, pts, g):
    from paper_2102_08514_b300.binding import interp_backward
    v = itp.eval(pts)
    v2, gr = itp.eval_grad(pts)
    dp = torch.empty_like(gr)
    interp_backward(itp.handle, pts, g, None, dp)
    torch.cuda.synchronize()
    return v, v2, gr, dp


@pytest.mark.parametrize("name", list(CASES))
def test_presorted_equals_unsorted(name):
    # fcc_voronoi2 and bcc_voronoi1 do not take the pre-sort by default; forced, it must still agree
    n_axis, n = CASES[name]
    torch, itp, dims, _ = _setup(name, n_axis, 71)
    pts = torch.from_numpy(mixed_points(name, dims, n, 72)).cuda()
    pts[n // 3] = float("nan")                                   # a non-finite query sorts too
    g = torch.linspace(-1, 1, n, device="cuda")
    res = []
    for flag in ("1", "0"):
        itp.set_option("presort", int(flag))
        res.append(_run_all(torch, itp, pts, g))
    for a, b in zip(*res):
        assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
    assert torch.isnan(res[0][0][n // 3])


@pytest.mark.parametrize("name", ["bcc_voronoi2", "d4s_8dir"])
def test_presorted_adjoint(name):
    n_axis, _ = CASES[name]
    torch, itp, dims, _ = _setup(name, n_axis, 73)
    n = 100_003
    pts = torch.from_numpy(mixed_points(name, dims, n, 74)).cuda()
    g = torch.from_numpy(make_rng(75, 0).uniform(-1, 1, n).astype(np.float32)).cuda()
    out = []
    for flag in ("1", "0"):
        itp.set_option("presort", int(flag))
        dc, _ = itp.backward(pts, g)
        torch.cuda.synchronize()
        out.append(dc.clone())
    # the same FP32 terms summed by atomics in another order: each site's sum of at most ~n x
    # lookups / sites terms of size <= max|phi| |g|; rounding stays far below 1e-4 of the largest
    scale = out[1].abs().max().item()
    assert scale > 0
    assert (out[0] - out[1]).abs().max().item() <= 1e-4 * scale


def test_presorted_matches_oracle():
    # the forced pre-sort on a small BCC V_2 case, against the FP64 oracle
    name = "bcc_voronoi2"
    torch, itp, dims, c = _setup(name, 10, 76)
    lat = LATTICES[SPLINES[name].lattice]
    pts = mixed_points(name, dims, 397, 77)
    itp.set_option("presort", 1)
    v, gr = itp.eval_grad(torch.from_numpy(pts).cuda())
    ref_v, ref_g = OracleSpline(name).eval_sum(lat.D, lat.cosets, c.astype(np.float64), pts.astype(np.float64),
                                               grad=True)
    cm = np.abs(c).max()
    G = grad_bound(name, pts[::13].astype(np.float64))
    fin = np.isfinite(ref_v)
    assert np.abs(v.cpu().numpy()[fin] - ref_v[fin]).max() <= VALUE_TOL * cm
    assert np.abs(gr.cpu().numpy()[fin] - ref_g[fin]).max() <= VALUE_TOL * cm * G


def test_presort_skipped_under_graph_capture():
    # a captured call cannot take scratch from the pool: it runs the binned kernel unsorted, with
    # the same results as the eager (pre-sorted) call
    name = "bcc_voronoi2"
    torch, itp, dims, _ = _setup(name, 12, 78)
    lo, hi = interior_box(name, dims)
    n = 1 << 17
    pts = torch.from_numpy(uniform_points(make_rng(79, 0), n, lo, hi)).cuda()
    eager = itp.eval(pts)
    out = torch.empty(n, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        itp.eval(pts, out)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        itp.eval(pts, out)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)


def test_presorted_host_path():
    # interp_eval_host: chunks of 2^20 (pre-sorted) plus a ragged tail below 2^16 (unsorted)
    torch = require_cuda()
    from paper_2102_08514_b300.binding import interp_eval_host
    name = "bcc_voronoi2"
    torch, itp, dims, _ = _setup(name, 12, 80)
    lo, hi = interior_box(name, dims)
    n = (2 << 20) + 777
    pts = torch.from_numpy(uniform_points(make_rng(81, 0), n, lo, hi)).pin_memory()
    out = torch.empty(n, pin_memory=True)
    grad = torch.empty(n, 3, pin_memory=True)
    interp_eval_host(itp.handle, pts, out, grad)
    torch.cuda.synchronize()
    v, g = itp.eval_grad(pts.cuda())
    assert torch.equal(out, v.cpu()) and torch.equal(grad, g.cpu())


def test_presort_default_rule():
    # interp_info_t.presort: on where it measured faster (BCC V_2, D4), off elsewhere (D4*: slower)
    require_cuda()
    want = {"bcc_voronoi2": 1, "d4_8dir": 1, "d4s_8dir": 0, "bcc_voronoi1": 0, "fcc_voronoi2": 0, "bcc_quintic": 0}
    for name, w in want.items():
        itp = make_interpolator(name, (6,) * len(SPLINES[name].xi))
        assert itp.info.presort == w, name


def test_presorted_half_storage():
    # the pre-sort in front of the FP16-storage binned kernel (BCC V_1 keeps FP16 kernels)
    name = "bcc_voronoi1"
    torch = require_cuda()
    dims = (12, 12, 12)
    itp = make_interpolator(name, dims, "f16")
    lat = LATTICES[SPLINES[name].lattice]
    c = make_rng(82, 3).uniform(-1, 1, (len(lat.cosets),) + dims).astype(np.float32)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    pts = torch.from_numpy(mixed_points(name, dims, 70001, 83)).cuda()
    res = []
    for flag in ("1", "0"):
        itp.set_option("presort", int(flag))
        res.append(itp.eval_grad(pts))
    for a, b in zip(*res):
        assert torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0))
