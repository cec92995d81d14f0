"""Host logic of bench.py: the kernel launches a step claims (the evaluation kernel, the adjoint
kernel plus the unpadding add, and with the piece pre-sort six kernels per chunk of 2^22 queries
for the value forms, five plus the add for the adjoint) and when the pre-sort applies."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_launches_per_step():
    n = 1 << 24                                        # 4 chunks of 2^22
    assert bench.launches_per_step("value", n, False) == 1
    assert bench.launches_per_step("value_grad", n, False) == 1
    assert bench.launches_per_step("adjoint", n, False) == 2
    assert bench.launches_per_step("value", n, True) == 24
    assert bench.launches_per_step("value_grad", n + 1, True) == 30   # a fifth, ragged chunk
    assert bench.launches_per_step("adjoint", n, True) == 21
    assert bench.launches_per_step("adjoint", n, False, True) == 5


def test_adjoint_bins_apply(monkeypatch):
    # the library's rule for the binned adjoint (wide 3-D stencils, many queries)
    monkeypatch.delenv("INTERP_B300_ADJOINT_BINS", raising=False)
    quintic = types.SimpleNamespace(s=3, n_pieces=1, D=2, lookups_per_query=32.0, dims=(128, 128, 128, 1), halo=2,
                                    n_cosets=2)
    fcc = types.SimpleNamespace(s=3, n_pieces=3, D=2, lookups_per_query=16.0, dims=(128, 128, 128, 1), halo=1,
                                n_cosets=4)
    d4s = types.SimpleNamespace(s=4, n_pieces=6, D=2, lookups_per_query=60.0, dims=(48, 48, 48, 48), halo=2,
                                n_cosets=2)
    assert bench.adjoint_bins_apply(quintic, 1 << 24)
    assert not bench.adjoint_bins_apply(quintic, 1 << 16)
    assert not bench.adjoint_bins_apply(fcc, 1 << 24)
    assert not bench.adjoint_bins_apply(d4s, 1 << 24)
    monkeypatch.setenv("INTERP_B300_ADJOINT_BINS", "1")
    assert bench.adjoint_bins_apply(fcc, 10)


def test_presort_applies(monkeypatch):
    monkeypatch.delenv("INTERP_B300_PRESORT", raising=False)
    on = types.SimpleNamespace(presort=1, n_pieces=14, binned=1)
    off = types.SimpleNamespace(presort=0, n_pieces=6, binned=1)
    assert bench.presort_applies(on, 1 << 16) and not bench.presort_applies(on, (1 << 16) - 1)
    assert not bench.presort_applies(off, 1 << 24)
    monkeypatch.setenv("INTERP_B300_PRESORT", "1")
    assert bench.presort_applies(off, 10)
    assert not bench.presort_applies(types.SimpleNamespace(presort=0, n_pieces=1, binned=0), 1 << 24)
    assert not bench.presort_applies(types.SimpleNamespace(presort=0, n_pieces=4, binned=0), 1 << 24)
    monkeypatch.setenv("INTERP_B300_PRESORT", "0")
    assert not bench.presort_applies(on, 1 << 24)


def test_distinct_sectors_match_the_support():
    """The sector count walks the kernels' fold, piece and stencil; here the same count from the
    oracle's support instead: every coset site n with phi(x - n) != 0, bricked the same way."""
    import numpy as np
    import oracle
    from synth import LATTICES, SPLINES, WORKLOADS, interior_box, make_rng, uniform_points
    for wname in ("bcc_quintic_128", "fcc_6dir_128"):
        wl = WORKLOADS[wname]
        sp = SPLINES[wl.spline]
        lat = LATTICES[sp.lattice]
        xi = np.asarray(sp.xi)
        o = oracle.Spline(xi, abs(round(np.linalg.det(np.asarray(lat.L, dtype=float)))))
        D, M, H = lat.D, len(lat.cosets), 2 if wl.spline == "bcc_quintic" else 1
        lbs = [bench.brick_lb(3, 4, M, a) for a in range(3)]
        lo, hi = interior_box(wl.spline, wl.dims)
        pts = uniform_points(make_rng(7, 1), 24, lo, hi)
        grid = np.stack(np.meshgrid(*[np.arange(-3, 4)] * 3, indexing="ij"), -1).reshape(-1, 3)
        for x in pts.astype(np.float64):
            keys = set()
            for k, l in enumerate(lat.cosets):
                i = np.floor((x - l) / D).astype(np.int64) + grid
                val = o.phi(x - (D * i + np.asarray(l)))
                for ii in i[val != 0]:
                    P = ii + 2 * H
                    keys.add((k,) + tuple(int(P[a]) >> lbs[a] for a in range(3)))
            assert bench.distinct_sectors_per_query(wl.spline, x[None].astype(np.float32)) == len(keys), (wname, x)


def test_distinct_lines_match_the_support():
    """The 128-byte line count (the requests of the warp-cooperative gathers) from the oracle's
    support and the padded bricked layout written out: bricks of 2 x 2 x 2 FP32 sites in row-major
    order of the padded coset array (last axis fastest), cosets one after another, 4 bricks per
    line."""
    import numpy as np
    import oracle
    from synth import LATTICES, SPLINES, WORKLOADS, interior_box, make_rng, uniform_points
    wl = WORKLOADS["bcc_quintic_128"]
    sp = SPLINES[wl.spline]
    lat = LATTICES[sp.lattice]
    o = oracle.Spline(np.asarray(sp.xi), abs(round(np.linalg.det(np.asarray(lat.L, dtype=float)))))
    D, H = lat.D, 2
    nb = [(n + 4 * H + 1) // 2 for n in wl.dims]         # bricks per axis of the padded array
    lo, hi = interior_box(wl.spline, wl.dims)
    pts = uniform_points(make_rng(7, 2), 16, lo, hi)
    grid = np.stack(np.meshgrid(*[np.arange(-3, 4)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for x in pts.astype(np.float64):
        lines = set()
        for k, l in enumerate(lat.cosets):
            i = np.floor((x - l) / D).astype(np.int64) + grid
            val = o.phi(x - (D * i + np.asarray(l)))
            for ii in i[val != 0]:
                b = (ii + 2 * H) // 2
                lines.add((k * nb[0] * nb[1] * nb[2] + (b[0] * nb[1] + b[1]) * nb[2] + b[2]) // 4)
        got = bench.distinct_sectors_per_query(wl.spline, x[None].astype(np.float32), dims=wl.dims)
        assert got == len(lines), (x, got, len(lines))
