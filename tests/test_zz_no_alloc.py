"""interp_backward_noalloc: the adjoint for callers that cannot allocate device memory when they
call it (their host program owns the allocator, or they run under a fixed memory budget).  Its
scratch is a static device array inside the library, so this file checks, through the C ABI, that
two calls in a row give the same result as interp_backward (the array is cleared between calls),
and that a handle too large for the array is refused.  It is collected last on purpose."""
import numpy as np
import pytest

from synth import LATTICES, SPLINES, interior_box, make_rng, uniform_points

pytestmark = pytest.mark.gpu


def _setup(name, dims, seed):
    import torch
    from paper_2102_08514_b300.binding import Interpolator
    assert torch.cuda.is_available(), "GPU test"
    sp = SPLINES[name]
    lat = LATTICES[sp.lattice]
    itp = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), dims, "f32")
    c = make_rng(seed, 1).uniform(-1, 1, itp.shape).astype(np.float32)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    return torch, itp


def _case(torch, itp, name, dims, seed, n):
    lo, hi = interior_box(name, dims)
    pts = torch.from_numpy(uniform_points(make_rng(seed, 2), n, lo - 3, hi + 3)).cuda()
    g = torch.from_numpy(make_rng(seed, 3).uniform(-1, 1, n).astype(np.float32)).cuda()
    return pts, g


@pytest.mark.parametrize("name,dims", [("bcc_quintic", (12, 12, 12)), ("fcc_6dir", (10, 10, 10)),
                                       ("d4s_8dir", (6, 6, 6, 6))])
def test_noalloc_adjoint_matches_interp_backward_twice(name, dims):
    from paper_2102_08514_b300.binding import interp_backward, interp_backward_noalloc
    torch, itp = _setup(name, dims, 31)
    for call, seed in enumerate((41, 42)):          # two calls in a row: stale scratch must not leak
        pts, g = _case(torch, itp, name, dims, seed, 3001 + 500 * call)
        ref = torch.zeros(itp.shape, device="cuda")
        interp_backward(itp.handle, pts, g, ref)
        bound = torch.zeros(itp.shape, device="cuda")
        interp_backward(itp.handle, pts, g.abs(), bound)
        got = torch.zeros(itp.shape, device="cuda")
        dpts = torch.empty(pts.shape[0], itp.s, device="cuda")
        interp_backward_noalloc(itp.handle, pts, g, got, dpts)
        dref = torch.empty_like(dpts)
        interp_backward(itp.handle, pts, g, None, dref)
        torch.cuda.synchronize()
        # the adjoint tolerance of the parity tests (FP32 atomics in arbitrary order)
        assert bool(torch.all((got - ref).abs() <= 4e-6 * bound + 1e-7)), (call, float((got - ref).abs().max()))
        assert torch.equal(dpts, dref)


@pytest.mark.parametrize("presort", [-1, 1])
def test_noalloc_allocates_nothing_where_the_pullback_would_presort(presort):
    """BCC V_2 with 2^16 queries and dpts: interp_backward takes the piece pre-sort there (pool
    scratch), interp_backward_noalloc must not -- checked with the library's own allocation count,
    with the default options and with the pre-sort forced on for every call."""
    import torch
    from paper_2102_08514_b300.binding import (Interpolator, interp_backward, interp_backward_noalloc,
                                               interp_debug_device_allocations)
    name, dims = "bcc_voronoi2", (20, 20, 20)
    itp = Interpolator.named(name, dims)
    itp.set_option("presort", presort)
    itp.set_coeffs(torch.from_numpy(make_rng(7, 1).uniform(-1, 1, itp.shape).astype(np.float32)).cuda())
    n = 1 << 16
    pts, g = _case(torch, itp, name, dims, 8, n)
    ref = torch.zeros(itp.shape, device="cuda")
    dref = torch.empty(n, 3, device="cuda")
    interp_backward(itp.handle, pts, g, ref, dref)            # allocates its buffer and pool scratch
    bound = torch.zeros(itp.shape, device="cuda")
    interp_backward(itp.handle, pts, g.abs(), bound)
    got = torch.zeros(itp.shape, device="cuda")
    dpts = torch.empty(n, 3, device="cuda")
    torch.cuda.synchronize()
    for _ in range(2):
        got.zero_()
        before = interp_debug_device_allocations()
        interp_backward_noalloc(itp.handle, pts, g, got, dpts)
        after = interp_debug_device_allocations()
        torch.cuda.synchronize()
        assert after == before
        assert bool(torch.all((got - ref).abs() <= 4e-6 * bound + 1e-7)), float((got - ref).abs().max())
        assert torch.equal(dpts, dref)


def test_noalloc_dpts_only_has_no_size_limit():
    from paper_2102_08514_b300.binding import interp_backward, interp_backward_noalloc
    torch, itp = _setup("cc_7dir", (208, 208, 208), 5)        # padded FP32 buffer > 8 Mi elements
    pts, g = _case(torch, itp, "cc_7dir", (208, 208, 208), 6, 1000)
    dpts = torch.empty(1000, 3, device="cuda")
    interp_backward_noalloc(itp.handle, pts, g, None, dpts)
    dref = torch.empty_like(dpts)
    interp_backward(itp.handle, pts, g, None, dref)
    torch.cuda.synchronize()
    assert torch.equal(dpts, dref)


def test_noalloc_refuses_handles_beyond_its_array():
    from paper_2102_08514_b300.binding import INTERP_ESIZE, InterpError, interp_backward_noalloc
    torch, itp = _setup("cc_7dir", (208, 208, 208), 5)        # padded FP32 buffer > 8 Mi elements
    pts, g = _case(torch, itp, "cc_7dir", (208, 208, 208), 6, 100)
    out = torch.zeros(itp.shape, device="cuda")
    with pytest.raises(InterpError) as e:
        interp_backward_noalloc(itp.handle, pts, g, out)
    assert e.value.status == INTERP_ESIZE
    assert float(out.abs().max()) == 0.0
