"""GPU: the D4 lattice (8 cosets) with Sec. 5.2's spline, the lattice prefilter (interp_prefilter)
against the oracle's world-grid prefilter, and Sec. 5.2's approximation experiment: a Gaussian
(sigma = 0.125) sampled on h L_D4, prefiltered, interpolated, L2 error over [-0.5, 0.5]^4 by Monte
Carlo with 10,000 samples, h halved repeatedly; the error falls by about 1/16 per halving once h
resolves the Gaussian (fourth order), by about 1/4 without the prefilter.
"""
import numpy as np
import pytest

import oracle
from synth import LATTICES, SPLINES, gaussian, make_rng

from _gpu_common import VALUE_TOL, OracleSpline, make_interpolator, mixed_points, require_cuda

pytestmark = pytest.mark.gpu


def _prefilter_parity(name, dims, taps, w, storage="f32"):
    torch = require_cuda()
    lat = LATTICES[SPLINES[name].lattice]
    itp = make_interpolator(name, dims, storage)
    f = make_rng(41, 0).uniform(-1, 1, (len(lat.cosets),) + tuple(dims)).astype(np.float32)
    itp.prefilter(torch.from_numpy(f).cuda(), taps, w)
    c_ref = oracle.prefilter(lat.L, lat.D, lat.cosets, f.astype(np.float64), taps, np.asarray(w, np.float64))
    pts = mixed_points(name, dims, 1500, 42)
    got = itp.eval(torch.from_numpy(pts).cuda()).cpu().numpy()
    ref = OracleSpline(name).eval_sum(lat.D, lat.cosets, c_ref, pts)
    # FP32 filter sums (weights rounded to FP32) plus the evaluation's own tolerance
    tol = VALUE_TOL * np.abs(c_ref).max() + 4e-7 * np.abs(np.asarray(w)).sum()
    return np.abs(got - ref).max(), tol


def test_prefilter_d4_quasi_interpolation():
    from paper_2102_08514_b300.binding import d4_quasi_interpolation_filter
    taps, w = d4_quasi_interpolation_filter()
    err, tol = _prefilter_parity("d4_8dir", (5, 6, 4, 7), taps, w)
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_prefilter_any_lattice_filter(storage):
    # a filter on BCC: the origin and the 8 nearest sites (+-1, +-1, +-1)
    taps = np.array([(0, 0, 0)] + [(a, b, c) for a in (1, -1) for b in (1, -1) for c in (1, -1)], np.int32)
    w = np.array([2.0] + [-0.125] * 8, np.float32)
    err, tol = _prefilter_parity("bcc_quintic", (9, 8, 10), taps, w, storage)
    if storage == "f16":
        tol += 2.0 ** -11 * 3.0        # the coefficients are rounded to binary16
    assert err <= tol, (err, tol)


def test_prefilter_rejects_non_lattice_taps():
    torch = require_cuda()
    from paper_2102_08514_b300.binding import InterpError
    itp = make_interpolator("d4_8dir", (4, 4, 4, 4))
    f = torch.zeros(itp.shape, device="cuda")
    with pytest.raises(InterpError):
        itp.prefilter(f, np.array([[1, 0, 0, 0]], np.int32), np.array([1.0], np.float32))   # odd sum
    with pytest.raises(InterpError):
        itp.prefilter(f, np.zeros((65, 4), np.int32), np.ones(65, np.float32))              # too many taps


def _d4_experiment(torch, j, Y, prefilter=True):
    """L2 error over the Monte Carlo points Y (world coordinates) at h = 0.5 / 2^j."""
    from paper_2102_08514_b300.binding import Interpolator, d4_quasi_interpolation_filter
    lat = LATTICES["d4"]
    h = 0.5 / 2 ** j
    q = 2 ** j + 6                   # lattice point (q, q, q, q) sits at the world origin
    N = 2 ** j + 7                   # sites reach 5 lattice units (stencil 4 + filter 1) past the domain
    itp = Interpolator.named("d4_8dir", (N,) * 4)
    # samples of the separable Gaussian at the sites 2 i + l_k (world h (2 i + l_k - q)), built on
    # the device as outer products
    i = torch.arange(N, device="cuda", dtype=torch.float64)
    f = torch.empty(itp.shape, device="cuda", dtype=torch.float32)
    for k, lk in enumerate(lat.cosets):
        fac = [torch.exp(-(h * (2 * i + lk[a] - q)) ** 2 / (2 * 0.125 ** 2)) for a in range(4)]
        f[k] = torch.einsum("a,b,c,d->abcd", *fac).float()
    if prefilter:
        taps, w = d4_quasi_interpolation_filter()
        itp.prefilter(f, taps, w)
    else:
        itp.set_coeffs(f)
    x = torch.from_numpy((Y / h + q).astype(np.float32)).cuda()
    v = itp.eval(x).double().cpu().numpy()
    return float(np.sqrt(np.mean((v - gaussian(Y)) ** 2)))


def test_d4_convergence_experiment():
    torch = require_cuda()
    Y = make_rng(56, 0).uniform(-0.5, 0.5, (10_000, 4))
    errs, plain = [], []
    for j in range(7):
        errs.append(_d4_experiment(torch, j, Y))
        plain.append(_d4_experiment(torch, j, Y, prefilter=False))
    print("\nSec. 5.2 D4 experiment: j, h, L2 error (prefiltered), ratio, L2 error (no prefilter), ratio")
    for j in range(7):
        r = errs[j - 1] / errs[j] if j else float("nan")
        rp = plain[j - 1] / plain[j] if j else float("nan")
        print(f"  {j} {0.5 / 2 ** j:.6f} {errs[j]:.3e} {r:6.2f} {plain[j]:.3e} {rp:6.2f}")
    # fourth order once h resolves the Gaussian (the 1/16 per halving of Sec. 5.2)
    assert 12.0 < errs[4] / errs[5] < 20.0 and 12.0 < errs[5] / errs[6] < 20.0
    # second order without the prefilter
    assert 3.0 < plain[5] / plain[6] < 5.0
