"""Lattices, splines and seeded inputs shaped like the paper's workloads.

Frame: the paper's integer frame (Sec. 3).  The BCC lattice is {all coordinates of equal parity}
(L_BCC of Sec. 3), the FCC lattice {even coordinate sum} (L_FCC), D4* = 2Z^4 u (2Z^4 + (1,1,1,1)).
Each is stored as Cartesian cosets D Z^s + l_k (Sec. 4.1, Fig. 2) with D = 2 (D = 1 for CC).

The paper renders the Marschner-Lobb function (Sec. 5.1); the closed-form signal below is the one
the workloads use in its place, sampled at the lattice sites.  No dataset is read.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["LatticeSpec", "SplineSpec", "LATTICES", "SPLINES", "Workload", "WORKLOADS",
           "interior_box", "make_rng", "uniform_points", "coefficients", "marschner_lobb", "gaussian", "D4_GAUSS_SIGMA",
           "site_positions", "ray_setup", "ray_points", "batch_volumes", "hashed_coefficients"]

SEED_BASE = 2102


@dataclass(frozen=True)
class LatticeSpec:
    name: str
    L: tuple          # generating matrix (rows)
    D: int            # coset grid spacing
    cosets: tuple     # coset shifts l_k


@dataclass(frozen=True)
class SplineSpec:
    name: str
    lattice: str
    xi: tuple         # s x n direction matrix (rows); for a Voronoi spline, 2 G (see order)
    order: int = 0    # 0: box spline M_xi; n >= 1: Voronoi spline V_n of the lattice, whose Voronoi
                      # region is the centred zonotope of the generators G = xi / 2


LATTICES = {
    "cc": LatticeSpec("cc", ((1, 0, 0), (0, 1, 0), (0, 0, 1)), 1, ((0, 0, 0),)),
    # Sec. 3 L_BCC; two cosets, the second shifted by (1,1,1) (Sec. 4.1)
    "bcc": LatticeSpec("bcc", ((-1, 1, 1), (1, -1, 1), (1, 1, -1)), 2, ((0, 0, 0), (1, 1, 1))),
    # Sec. 3 L_FCC; four cosets (Fig. 1)
    "fcc": LatticeSpec("fcc", ((0, 1, 1), (1, 0, 1), (1, 1, 0)), 2,
                       ((0, 0, 0), (0, 1, 1), (1, 0, 1), (1, 1, 0))),
    # D4* in the integer frame: all coordinates of equal parity (Sec. 5.2 mentions D4*)
    "d4s": LatticeSpec("d4s", ((2, 0, 0, 1), (0, 2, 0, 1), (0, 0, 2, 1), (0, 0, 0, 1)), 2,
                       ((0, 0, 0, 0), (1, 1, 1, 1))),
    # Sec. 5.2 L_D4: even coordinate sum, eight cosets of 2Z^4 (the points of {0,1}^4 of even sum)
    "d4": LatticeSpec("d4", ((-1, 0, 0, 0), (1, 0, -1, -1), (0, -1, 0, 1), (0, -1, 1, 0)), 2,
                      ((0, 0, 0, 0), (0, 0, 1, 1), (0, 1, 0, 1), (0, 1, 1, 0), (1, 0, 0, 1), (1, 0, 1, 0),
                       (1, 1, 0, 0), (1, 1, 1, 1))),
}

_BCC_RD = ((-1, 1, 1, -1), (1, -1, 1, -1), (1, 1, -1, -1))
_BCC_VOR = ((1, 1, 1, 1, 0, 0), (1, -1, 0, 0, 1, 1), (0, 0, 1, -1, 1, -1))
_FCC_VOR = ((1, 1, -1, -1), (1, -1, 1, -1), (1, -1, -1, 1))
SPLINES = {
    # Table 1: linear rhombic dodecahedron on BCC (4 directions)
    "bcc_linear": SplineSpec("bcc_linear", "bcc", _BCC_RD),
    # Table 1: quintic rhombic dodecahedron on BCC (the 4 directions twice)
    "bcc_quintic": SplineSpec("bcc_quintic", "bcc", tuple(r + r for r in _BCC_RD)),
    # Table 1: cubic truncated octahedron on FCC (6 directions)
    "fcc_6dir": SplineSpec("fcc_6dir", "fcc", ((1, -1, 1, 1, 0, 0), (1, 1, 0, 0, 1, -1),
                                              (0, 0, 1, -1, 1, 1))),
    # Table 1: truncated rhombic dodecahedron on CC (7 directions)
    "cc_7dir": SplineSpec("cc_7dir", "cc", ((1, 0, 0, -1, 1, 1, -1), (0, 1, 0, 1, -1, 1, -1),
                                           (0, 0, 1, 1, 1, -1, -1))),
    # Sec. 5.2: the 8 directions (1, +-1, +-1, +-1)
    "d4s_8dir": SplineSpec("d4s_8dir", "d4s", ((1, 1, 1, 1, 1, 1, 1, 1),
                                               (1, 1, 1, 1, -1, -1, -1, -1),
                                               (1, 1, -1, -1, 1, 1, -1, -1),
                                               (1, -1, 1, -1, 1, -1, 1, -1))),
    # Sec. 5.2: the same 8 directions on D4 (240 lookups)
    "d4_8dir": SplineSpec("d4_8dir", "d4", ((1, 1, 1, 1, 1, 1, 1, 1),
                                             (1, 1, 1, 1, -1, -1, -1, -1),
                                             (1, 1, -1, -1, 1, 1, -1, -1),
                                             (1, -1, 1, -1, 1, -1, 1, -1))),
    # Table 1: quartic truncated rhombic dodecahedron on BCC (7 directions)
    "bcc_quartic": SplineSpec("bcc_quartic", "bcc", ((2, 0, 0, -1, 1, 1, -1), (0, 2, 0, 1, -1, 1, -1),
                                                     (0, 0, 2, 1, 1, -1, -1))),
    # Table 1: linear rhombic dodecahedron on CC
    "cc_linear_rd": SplineSpec("cc_linear_rd", "cc", _BCC_RD),
    # Table 1: CC Voronoi splines 1-3 (the identity directions repeated 2, 3, 4 times)
    "cc_voronoi1": SplineSpec("cc_voronoi1", "cc", tuple(r * 2 for r in ((1, 0, 0), (0, 1, 0), (0, 0, 1)))),
    "cc_voronoi2": SplineSpec("cc_voronoi2", "cc", tuple(r * 3 for r in ((1, 0, 0), (0, 1, 0), (0, 0, 1)))),
    "cc_voronoi3": SplineSpec("cc_voronoi3", "cc", tuple(r * 4 for r in ((1, 0, 0), (0, 1, 0), (0, 0, 1)))),
    # Table 1: Voronoi splines V_1, V_2 on BCC (truncated octahedron, six generators
    # (+-1, +-1, 0) / 2) and on FCC (rhombic dodecahedron, four generators (+-1, +-1, +-1) / 2)
    "bcc_voronoi1": SplineSpec("bcc_voronoi1", "bcc", _BCC_VOR, 1),
    "bcc_voronoi2": SplineSpec("bcc_voronoi2", "bcc", _BCC_VOR, 2),
    "fcc_voronoi1": SplineSpec("fcc_voronoi1", "fcc", _FCC_VOR, 1),
    "fcc_voronoi2": SplineSpec("fcc_voronoi2", "fcc", _FCC_VOR, 2),
}


def support_halfwidth(xi) -> np.ndarray:
    """Half-width per axis of the bounding box of the centred support (input placement only)."""
    return np.abs(np.asarray(xi)).sum(axis=1) / 2.0


def interior_box(spline: str, dims) -> tuple[np.ndarray, np.ndarray]:
    """Points strictly inside this box touch only stored coefficient sites (every coset)."""
    sp = SPLINES[spline]
    lat = LATTICES[sp.lattice]
    # a Voronoi spline V_n is supported on (n+1) times the Voronoi region, the zonotope of xi / 2
    h = support_halfwidth(sp.xi) * ((sp.order + 1) / 2 if sp.order else 1)
    cos = np.asarray(lat.cosets)
    lo = cos.max(axis=0) + h - lat.D
    hi = cos.min(axis=0) + lat.D * np.asarray(dims) - h
    return lo.astype(np.float64), hi.astype(np.float64)


@dataclass(frozen=True)
class Workload:
    name: str
    spline: str
    dims: tuple        # N per axis of every coset array
    coeffs: str        # "uniform" | "normal" | "signal"
    queries: int
    seed: int


WORKLOADS = {
    # correctness / latency case: 2 x 16^3 FP64 coefficients, 10^4 queries, value only
    "bcc_linear_16": Workload("bcc_linear_16", "bcc_linear", (16, 16, 16), "uniform", 10_000, SEED_BASE + 0),
    # headline case: 2 x 128^3 FP32 samples of the test signal, 2^24 random queries
    "bcc_quintic_128": Workload("bcc_quintic_128", "bcc_quintic", (128, 128, 128), "signal", 1 << 24, SEED_BASE + 1),
    # fitting case: 4 x 128^3, 2^22 samples
    "fcc_6dir_128": Workload("fcc_6dir_128", "fcc_6dir", (128, 128, 128), "signal", 1 << 22, SEED_BASE + 2),
    # precision case: CC 256^3 Gaussian coefficients, 2^24 queries
    "cc_7dir_256": Workload("cc_7dir_256", "cc_7dir", (256, 256, 256), "normal", 1 << 24, SEED_BASE + 3),
    # 4-D case: 2 x 48^4, 2^24 queries
    "d4s_8dir_48": Workload("d4s_8dir_48", "d4s_8dir", (48, 48, 48, 48), "uniform", 1 << 24, SEED_BASE + 4),
}


# Sec. 5.2's approximation experiment: a Gaussian with mean 0 and sigma = 0.125 on [-0.5, 0.5]^4,
# sampled on the scaled lattice h L_D4 for h = 0.5 / 2^j
D4_GAUSS_SIGMA = 0.125


def gaussian(p: np.ndarray, sigma: float = D4_GAUSS_SIGMA) -> np.ndarray:
    """exp(-|p|^2 / (2 sigma^2)) (unnormalised) at points p (..., s)."""
    return np.exp(-(np.asarray(p, dtype=np.float64) ** 2).sum(axis=-1) / (2.0 * sigma * sigma))


def make_rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.default_rng([seed, stream])


def uniform_points(rng: np.random.Generator, n: int, lo, hi) -> np.ndarray:
    """n FP32 points uniform in the box [lo, hi] (rows)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    u = rng.random((n, lo.size))
    return (lo + u * (hi - lo)).astype(np.float32)


def marschner_lobb(p: np.ndarray) -> np.ndarray:
    """rho(x,y,z) = (1 - sin(pi z/2) + 0.25 (1 + cos(12 pi cos(pi r/2)))) / 2.5, r = sqrt(x^2+y^2),
    on [-1,1]^3 (the Marschner-Lobb test function the paper renders, Sec. 5.1)."""
    x, y, z = p[..., 0], p[..., 1], p[..., 2]
    r = np.sqrt(x * x + y * y)
    return (1.0 - np.sin(np.pi * z / 2.0) + 0.25 * (1.0 + np.cos(12.0 * np.pi * np.cos(np.pi * r / 2.0)))) / 2.5


def site_positions(lattice: str, dims) -> np.ndarray:
    """World positions D*i + l_k of every stored site, shape (M, *dims, s)."""
    lat = LATTICES[lattice]
    s = len(dims)
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    base = np.stack(grids, axis=-1) * lat.D
    return np.stack([base + np.asarray(l) for l in lat.cosets], axis=0).astype(np.float64)


def coefficients(wl: Workload, dtype=np.float32) -> np.ndarray:
    """Coefficient arrays, shape (M, *dims), coset-major, last axis fastest."""
    lat = LATTICES[SPLINES[wl.spline].lattice]
    shape = (len(lat.cosets),) + tuple(wl.dims)
    rng = make_rng(wl.seed, 1)
    if wl.coeffs == "uniform":
        c = rng.uniform(-1.0, 1.0, shape)
    elif wl.coeffs == "normal":
        c = rng.standard_normal(shape)
    elif wl.coeffs == "signal":
        # site at world w -> physical p = -1 + w / (D N / 2) per axis, covering [-1, 1)
        pos = site_positions(lat.name, wl.dims)
        p = -1.0 + pos / (lat.D * np.asarray(wl.dims) / 2.0)
        c = marschner_lobb(p)
    else:
        raise ValueError(wl.coeffs)
    return c.astype(dtype)


def hashed_coefficients(k, idx, xp=np):
    """Coefficient of coset k at integer site indices idx = (i_1, ..., i_s) (broadcastable int64
    arrays of numpy, or of torch when xp is torch): an integer hash of the indices mapped to
    multiples of 1/1024 in [-1, 1).  Exact in FP32 and computable for any slab of a volume too
    large to generate at once; the same values from numpy and torch."""
    mult = (73856093, 19349663, 83492791, 2654435761)
    h = k * 40503
    for a, i in enumerate(idx):
        h = h ^ (i * mult[a])
    if xp is np:
        return ((np.asarray(h) & 2047) - 1024).astype(np.float32) / np.float32(1024.0)
    return ((h & 2047) - 1024).to(xp.float32) / 1024.0


# ----------------------------------------------------------------------------- rays

def ray_setup(spline: str, dims, width: int = 1024, height: int = 1024, steps: int = 256):
    """Orthographic rays along d = normalize(3,2,1) through the interior box (an oblique
    direction, so that no lattice axis is favoured, Sec. 5.1).  Returns origin o, direction d,
    image-plane axes (e_u, e_v), pixel pitch and the box.  Each ray marches `steps` equal steps
    over its own chord of the box."""
    lo, hi = interior_box(spline, dims)
    centre = (lo + hi) / 2.0
    d = np.array([3.0, 2.0, 1.0])
    d /= np.linalg.norm(d)
    eu = np.cross(d, [0.0, 0.0, 1.0])
    eu /= np.linalg.norm(eu)
    ev = np.cross(d, eu)
    corners = np.array([[lo[0] if i & 1 else hi[0], lo[1] if i & 2 else hi[1], lo[2] if i & 4 else hi[2]]
                        for i in range(8)]) - centre
    ru = np.abs(corners @ eu).max()
    rv = np.abs(corners @ ev).max()
    return dict(centre=centre, d=d, eu=eu, ev=ev, half_u=ru, half_v=rv, lo=lo, hi=hi,
                width=width, height=height, steps=steps)


def ray_points(setup: dict, pixels: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Sample points (FP64) of the rays through the given pixel indices (n, 2) = (px, py):
    the chord of each ray with the box, split into `steps` equal steps at the step midpoints.
    Returns (points (n, steps, 3), valid (n,))."""
    c, d, eu, ev = setup["centre"], setup["d"], setup["eu"], setup["ev"]
    lo, hi = setup["lo"], setup["hi"]
    W, H, S = setup["width"], setup["height"], setup["steps"]
    u = (2.0 * (pixels[:, 0] + 0.5) / W - 1.0) * setup["half_u"]
    v = (2.0 * (pixels[:, 1] + 0.5) / H - 1.0) * setup["half_v"]
    o = c + u[:, None] * eu + v[:, None] * ev
    with np.errstate(divide="ignore", invalid="ignore"):
        t1 = (lo - o) / d
        t2 = (hi - o) / d
    tmin = np.minimum(t1, t2).max(axis=1)
    tmax = np.maximum(t1, t2).min(axis=1)
    valid = tmax > tmin
    dt = (tmax - tmin) / S
    ts = tmin[:, None] + (np.arange(S)[None, :] + 0.5) * dt[:, None]
    pts = o[:, None, :] + ts[..., None] * d
    return pts, valid


# ----------------------------------------------------------------------------- batched volumes

def batch_volumes(n_volumes: int = 64, seed: int = SEED_BASE + 4):
    """Volume v uses spline v mod 4 of (bcc_linear, bcc_quintic, fcc_6dir, cc_7dir); edge lengths
    per axis log-uniform in [32, 256]."""
    rng = make_rng(seed, 7)
    names = ("bcc_linear", "bcc_quintic", "fcc_6dir", "cc_7dir")
    out = []
    for v in range(n_volumes):
        dims = tuple(int(round(np.exp(rng.uniform(np.log(32), np.log(256))))) for _ in range(3))
        out.append((names[v % 4], dims))
    return out
