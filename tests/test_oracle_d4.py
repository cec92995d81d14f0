"""Pins of the oracle's D4 pieces (Sec. 5.2): the lattice, the 8-direction spline on it and the
quasi-interpolation prefilter.

* the prefilter's world-grid computation equals the definition c(n) = sum_t w_t f(n + v_t) summed
  site by site through a dictionary of world positions;
* with the prefilter, the spline reproduces cubic polynomials exactly (the filter inverts the
  spline's symbol to fourth order, which is what gives the error decay by 1/16 per halving of h
  that Sec. 5.2 reports); without it, quadratics are not reproduced;
* the filter's weights sum to one (7/3 - 24/18), and the D4 lattice has 8 cosets of 2Z^4.
"""
import numpy as np

import oracle
from synth import LATTICES, SPLINES, make_rng


def _d4():
    lat = LATTICES["d4"]
    return lat, oracle.Spline(np.asarray(SPLINES["d4_8dir"].xi), 2)


def test_d4_lattice_and_filter_weights():
    lat, _ = _d4()
    assert abs(round(np.linalg.det(np.asarray(lat.L, float)))) == 2
    sites = oracle.lattice_sites(lat.L, [0] * 4, [1] * 4)          # the coset shifts are the sites in {0,1}^4
    assert sorted(map(tuple, sites)) == sorted(map(tuple, lat.cosets))
    taps, w = oracle.d4_quasi_interpolation_taps()
    assert len(taps) == 25 and abs(w.sum() - 1) < 1e-15
    assert np.all((taps[1:] ** 2).sum(axis=1) == 2)


def test_prefilter_equals_the_sitewise_definition():
    lat, _ = _d4()
    dims = (4, 5, 3, 4)
    f = make_rng(31, 0).uniform(-1, 1, (8,) + dims)
    taps, w = oracle.d4_quasi_interpolation_taps()
    got = oracle.prefilter(lat.L, lat.D, lat.cosets, f, taps, w)
    world = {}
    for k, lk in enumerate(lat.cosets):
        for i in np.ndindex(*dims):
            world[tuple(2 * np.asarray(i) + np.asarray(lk))] = f[(k,) + i]
    for k, lk in enumerate(lat.cosets):
        for i in np.ndindex(*dims):
            n = 2 * np.asarray(i) + np.asarray(lk)
            ref = sum(wt * world.get(tuple(n + v), 0.0) for v, wt in zip(taps, w))
            assert abs(got[(k,) + i] - ref) < 1e-14


def _cubic(rng, centre, scale):
    alphas = [a for a in np.ndindex(4, 4, 4, 4) if sum(a) <= 3]
    coef = rng.uniform(-1, 1, len(alphas))

    def p(x):
        u = (np.asarray(x, dtype=np.float64) - centre) / scale
        return sum(c * np.prod(u ** np.asarray(a), axis=-1) for c, a in zip(coef, alphas))
    return p


def test_prefiltered_spline_reproduces_cubics():
    lat, spl = _d4()
    N = 8
    dims = (N,) * 4
    rng = make_rng(33, 0)
    p = _cubic(rng, centre=N - 0.5, scale=4.0)
    sites = np.stack([2 * np.stack(np.meshgrid(*[np.arange(N)] * 4, indexing="ij"), -1) + np.asarray(lk)
                      for lk in lat.cosets])
    f = p(sites)
    taps, w = oracle.d4_quasi_interpolation_taps()
    c = oracle.prefilter(lat.L, lat.D, lat.cosets, f, taps, w)
    # every stencil site (support half-width 4) and its filter neighbours (reach 1) are stored
    x = np.round(rng.uniform(5.0, 2 * N - 6.0, (16, 4)) * 256) / 256
    got = oracle.eval_sum(spl, lat.D, lat.cosets, c, x)
    assert np.abs(got - p(x)).max() < 1e-10
    # the spline alone (c = samples) smooths: it does not reproduce a quadratic
    q = lambda y: (((np.asarray(y) - (N - 0.5)) / 4.0) ** 2).sum(axis=-1)
    plain = oracle.eval_sum(spl, lat.D, lat.cosets, q(sites), x)
    assert np.abs(plain - q(x)).max() > 1e-2
