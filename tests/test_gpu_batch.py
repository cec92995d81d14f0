"""Batched evaluation (one persistent launch per dimension, CUDA graph, autotuned tiles) against
the per-handle path and the oracle."""
import numpy as np
import pytest

import oracle
from synth import LATTICES, SPLINES, interior_box, make_rng, uniform_points

from _gpu_common import VALUE_TOL, require_cuda

pytestmark = pytest.mark.gpu


def _volumes(seed, n):
    """Mixed splines (the four 3-D ones and the 4-D one), uneven sizes, ragged query counts."""
    rng = make_rng(seed, 0)
    names = ["bcc_linear", "bcc_quintic", "fcc_6dir", "cc_7dir", "d4s_8dir"]
    vols = []
    for v in range(n):
        name = names[v % len(names)]
        s = len(SPLINES[name].xi)
        dims = tuple(int(x) for x in rng.integers(5, 9 if s == 4 else 17, s))
        nq = int(rng.integers(1, 2500)) if v != 3 else 0            # one empty volume
        vols.append((name, dims, nq))
    return vols


def test_batch_matches_per_volume_eval_and_oracle():
    torch = require_cuda()
    from paper_2102_08514_b300.binding import Batch, Interpolator
    items, data = [], []
    for v, (name, dims, nq) in enumerate(_volumes(77, 13)):
        sp = SPLINES[name]
        lat = LATTICES[sp.lattice]
        itp = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), dims, "f32")
        c = make_rng(100 + v, 1).uniform(-1, 1, itp.shape).astype(np.float32)
        itp.set_coeffs(torch.from_numpy(c).cuda())
        lo, hi = interior_box(name, dims)
        pts = uniform_points(make_rng(200 + v, 2), nq, lo - 1.0, hi + 1.0)
        dp = torch.from_numpy(pts).cuda().reshape(nq, len(dims))
        out = torch.full((nq,), float("nan"), device="cuda")
        items.append((itp, dp, out))
        data.append((name, lat, c, pts))
    batch = Batch(items)
    tiles = batch.autotune()
    assert all(t % 128 == 0 and t >= 256 for t in tiles.values())
    for rep in range(2):                                      # graph replay
        for _, _, out in items:
            out.fill_(float("nan"))
        batch.run()
        torch.cuda.synchronize()
        for (itp, dp, out), (name, lat, c, pts) in zip(items, data):
            if dp.shape[0] == 0:
                continue
            ref = itp.eval(dp)
            assert torch.allclose(out, ref, rtol=0, atol=VALUE_TOL * float(np.abs(c).max())), name
    # spot check a few volumes against the oracle
    for (itp, dp, out), (name, lat, c, pts) in list(zip(items, data))[:6]:
        if len(pts) == 0:
            continue
        k = min(200, len(pts))
        o = oracle.Spline(np.asarray(SPLINES[name].xi), abs(round(np.linalg.det(np.asarray(lat.L, float)))))
        ref = oracle.eval_sum(o, lat.D, lat.cosets, c.astype(np.float64), pts[:k].astype(np.float64))
        assert np.abs(out[:k].cpu().numpy() - ref).max() <= VALUE_TOL * np.abs(c).max(), name


def test_batch_rejects_half_storage_and_bad_tiles():
    torch = require_cuda()
    from paper_2102_08514_b300.binding import (Batch, INTERP_EINVAL, INTERP_EUNSUPPORTED, InterpError,
                                               Interpolator, interp_batch_set_tile)
    sp = SPLINES["bcc_quintic"]
    lat = LATTICES["bcc"]
    h16 = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), (8, 8, 8), "f16")
    p = torch.zeros(10, 3, device="cuda")
    o = torch.zeros(10, device="cuda")
    with pytest.raises(InterpError) as e:
        Batch([(h16, p, o)])
    assert e.value.status == INTERP_EUNSUPPORTED
    h32 = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), (8, 8, 8), "f32")
    b = Batch([(h32, p, o)])
    with pytest.raises(InterpError) as e:
        interp_batch_set_tile(b._b, "bcc_quintic", 100)
    assert e.value.status == INTERP_EINVAL
    b.set_tiles({"bcc_quintic": 256})
    assert b.tiles() == {"bcc_quintic": 256}


def test_batch_with_handles_outside_the_persistent_kernel():
    # splines outside the persistent kernel's list (many-piece or heavy 3-D splines, 4-D) run their
    # own evaluation launch inside the same graph; a batch mixing both groups equals the
    # per-handle path, and only the persistent kernel's splines report a tile
    torch = require_cuda()
    from paper_2102_08514_b300.binding import Batch
    from _gpu_common import make_interpolator
    names = ["bcc_voronoi1", "bcc_quintic", "cc_voronoi3", "fcc_voronoi2", "d4_8dir", "cc_7dir"]
    items, cs = [], []
    for v, name in enumerate(names):
        s = len(SPLINES[name].xi)
        dims = (6,) * 4 if s == 4 else (9, 10, 11)
        itp = make_interpolator(name, dims)
        c = make_rng(300 + v, 1).uniform(-1, 1, itp.shape).astype(np.float32)
        itp.set_coeffs(torch.from_numpy(c).cuda())
        lo, hi = interior_box(name, dims)
        nq = 700 + 37 * v
        pts = torch.from_numpy(uniform_points(make_rng(400 + v, 2), nq, lo, hi)).cuda()
        items.append((itp, pts, torch.full((nq,), float("nan"), device="cuda")))
        cs.append(c)
    batch = Batch(items)
    assert set(batch.tiles()) == {"bcc_quintic", "cc_7dir"}
    batch.run()
    torch.cuda.synchronize()
    for (itp, pts, out), c, name in zip(items, cs, names):
        ref = itp.eval(pts)
        assert torch.allclose(out, ref, rtol=0, atol=VALUE_TOL * float(np.abs(c).max())), name
