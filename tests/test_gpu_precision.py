"""Reduced-precision coefficient storage on the CC 7-direction workload (256^3, N(0,1)
coefficients, FP32 arithmetic): error against the FP64 oracle two ways -- on the dequantised
coefficients (must meet the FP32 tolerance) and on the original ones (bounded by the storage
unit roundoff) -- on sampled queries of the full 2^24-query launch."""
import numpy as np
import pytest

import oracle
from synth import LATTICES, SPLINES, WORKLOADS, coefficients, interior_box, make_rng, uniform_points

from _gpu_common import VALUE_TOL, require_cuda

pytestmark = pytest.mark.gpu


def test_precision_report_cc_7dir_256():
    torch = require_cuda()
    from paper_2102_08514_b300.binding import Interpolator
    wl = WORKLOADS["cc_7dir_256"]
    sp = SPLINES[wl.spline]
    lat = LATTICES[sp.lattice]
    c = coefficients(wl)
    lo, hi = interior_box(wl.spline, wl.dims)
    pts = uniform_points(make_rng(wl.seed, 0), wl.queries, lo, hi)
    dp = torch.from_numpy(pts).cuda()
    idx = make_rng(wl.seed, 9).choice(wl.queries, 2048, replace=False)
    o = oracle.Spline(np.asarray(sp.xi), 1)
    P = pts[idx].astype(np.float64)
    ref = oracle.eval_sum(o, lat.D, lat.cosets, c.astype(np.float64), P)
    cmax = float(np.abs(c).max())
    report = {}
    for storage, tdt, unit in (("f32", torch.float32, 2.0 ** -24), ("f16", torch.float16, 2.0 ** -11),
                               ("bf16", torch.bfloat16, 2.0 ** -8)):
        itp = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), wl.dims, storage)
        cq = torch.from_numpy(c).to(tdt)
        itp.set_coeffs(cq.cuda())
        got = itp.eval(dp)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
        ref_q = ref if storage == "f32" else oracle.eval_sum(o, lat.D, lat.cosets, cq.double().numpy(), P)
        e_q, e_o = got - ref_q, got - ref
        report[storage] = dict(max_abs_vs_dequantised=np.abs(e_q).max(), rms_vs_dequantised=np.sqrt((e_q ** 2).mean()),
                               max_abs_vs_original=np.abs(e_o).max(), rms_vs_original=np.sqrt((e_o ** 2).mean()))
        assert np.abs(e_q).max() <= VALUE_TOL * cmax, (storage, report[storage])
        assert np.abs(e_o).max() <= 2 * unit * cmax + VALUE_TOL * cmax, (storage, report[storage])
        itp.close()
    print("\nprecision report, cc_7dir_256, max|c| = %.3f, 2048 sampled queries" % cmax)
    for k, v in report.items():
        print(k, " ".join(f"{a}={b:.3e}" for a, b in v.items()))
