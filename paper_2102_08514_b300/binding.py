"""Thin ctypes binding of the C ABI in include/interp.h (argument marshalling only).

Every computation runs in the CUDA kernels of libinterp_b300.so; this module only converts torch
tensors to device pointers and the current CUDA stream to a cudaStream_t.  If the library is
missing, loading fails loudly: there is no CPU or PyTorch fallback.

The functions carry the C names (interp_create, interp_eval, ...); ``Interpolator`` bundles a
handle with its tensors and ``LatticeInterp`` is the torch.autograd.Function whose backward is the
hand-written adjoint (interp_backward).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libinterp_b300.so")

INTERP_OK, INTERP_EINVAL, INTERP_EUNSUPPORTED, INTERP_ENOMEM, INTERP_ECUDA, INTERP_ESIZE = range(6)
INTERP_F32, INTERP_F16, INTERP_BF16, INTERP_F64 = range(4)

_lib = None


class InterpError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {_strerror(status)} (status {status})")


class InterpInfo(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int), ("n_cosets", ctypes.c_int), ("D", ctypes.c_int), ("halo", ctypes.c_int),
                ("n_pieces", ctypes.c_int), ("degree", ctypes.c_int), ("n_monomials", ctypes.c_int),
                ("dims", ctypes.c_int * 4), ("cosets", (ctypes.c_int32 * 4) * 8),
                ("lookups_per_query", ctypes.c_double), ("fma_value_per_query", ctypes.c_double),
                ("fma_grad_per_query", ctypes.c_double), ("coeff_count", ctypes.c_int64),
                ("name", ctypes.c_char_p), ("kind", ctypes.c_int), ("presort", ctypes.c_int),
                ("binned", ctypes.c_int), ("coop", ctypes.c_int)]


class Rays(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("du", ctypes.c_float * 3), ("dv", ctypes.c_float * 3),
                ("dir", ctypes.c_float * 3), ("box_lo", ctypes.c_float * 3), ("box_hi", ctypes.c_float * 3),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("steps", ctypes.c_int32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("vol", ctypes.c_void_p), ("pts", ctypes.c_void_p), ("npts", ctypes.c_int64),
                ("out", ctypes.c_void_p)]


def load(path: str = LIB_PATH):
    """Load libinterp_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run python -m paper_2102_08514_b300.build)")
    lib = ctypes.CDLL(path)
    P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.interp_strerror.argtypes = [I]
    lib.interp_strerror.restype = ctypes.c_char_p
    lib.interp_num_splines.restype = I
    lib.interp_spline_name.argtypes = [I]
    lib.interp_spline_name.restype = ctypes.c_char_p
    lib.interp_table_digest.restype = ctypes.c_char_p
    lib.interp_debug_device_allocations.argtypes = []
    lib.interp_debug_device_allocations.restype = ctypes.c_longlong
    lib.interp_create.argtypes = [I, P, P, I, P, I, ctypes.POINTER(ctypes.c_void_p)]
    lib.interp_create_named.argtypes = [ctypes.c_char_p, P, I, ctypes.POINTER(ctypes.c_void_p)]
    lib.interp_destroy.argtypes = [P]
    lib.interp_destroy.restype = None
    lib.interp_info.argtypes = [P, ctypes.POINTER(InterpInfo)]
    lib.interp_set_option.argtypes = [P, ctypes.c_char_p, I]
    lib.interp_get_option.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
    lib.interp_set_coeffs.argtypes = [P, P, I, I, P]
    lib.interp_prefilter.argtypes = [P, P, I, P, P, P]
    lib.interp_eval.argtypes = [P, P, I64, P, P]
    lib.interp_eval_grad.argtypes = [P, P, I64, P, P, P]
    lib.interp_backward.argtypes = [P, P, I64, P, P, P, P]
    lib.interp_debug_indices.argtypes = [P, P, I64, P, P, P]
    lib.interp_backward_noalloc.argtypes = [P, P, I64, P, P, P, P]
    lib.interp_sort_points.argtypes = [P, P, I64, P, P, P]
    lib.interp_sort_points.restype = I
    lib.interp_eval_host.argtypes = [P, P, I64, P, P, P]
    lib.interp_eval_host.restype = I
    lib.interp_eval_rays.argtypes = [P, ctypes.POINTER(Rays), I, P, P, P]
    lib.interp_eval_rays.restype = I
    lib.interp_batch_create.argtypes = [ctypes.POINTER(BatchItem), I, ctypes.POINTER(ctypes.c_void_p)]
    lib.interp_batch_autotune.argtypes = [P, P]
    lib.interp_batch_tile.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
    lib.interp_batch_set_tile.argtypes = [P, ctypes.c_char_p, I]
    lib.interp_batch_run.argtypes = [P, P]
    lib.interp_batch_destroy.argtypes = [P]
    lib.interp_batch_destroy.restype = None
    for f in (lib.interp_batch_create, lib.interp_batch_autotune, lib.interp_batch_tile, lib.interp_batch_set_tile,
              lib.interp_batch_run):
        f.restype = I
    for f in (lib.interp_set_option, lib.interp_get_option, lib.interp_create, lib.interp_create_named, lib.interp_info, lib.interp_prefilter, lib.interp_set_coeffs, lib.interp_eval, lib.interp_eval_grad,
              lib.interp_backward, lib.interp_debug_indices, lib.interp_backward_noalloc):
        f.restype = I
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return ["interp_strerror", "interp_num_splines", "interp_spline_name", "interp_table_digest",
            "interp_debug_device_allocations",
            "interp_create", "interp_create_named", "interp_destroy", "interp_prefilter", "interp_info",
            "interp_set_option", "interp_get_option", "interp_set_coeffs", "interp_eval",
            "interp_eval_grad", "interp_backward", "interp_debug_indices", "interp_backward_noalloc",
            "interp_batch_create", "interp_batch_autotune", "interp_batch_tile", "interp_batch_set_tile",
            "interp_batch_run", "interp_batch_destroy", "interp_eval_rays", "interp_eval_host",
            "interp_sort_points"]


def _strerror(st: int) -> str:
    try:
        return load().interp_strerror(st).decode()
    except Exception:  # library not loadable
        return "error"


def _check(st: int, what: str):
    if st != INTERP_OK:
        raise InterpError(st, what)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, name, dtype=None, device=True):
    if t is None:
        return None
    import torch
    if device and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def spline_names() -> list[str]:
    lib = load()
    return [lib.interp_spline_name(i).decode() for i in range(lib.interp_num_splines())]


def table_digest() -> str:
    return load().interp_table_digest().decode()


def interp_debug_device_allocations() -> int:
    """Device allocation calls the library has made in this process so far."""
    return int(load().interp_debug_device_allocations())


# ----------------------------------------------------------------------------- C-named wrappers

def interp_create_named(name: str, dims, storage: int = INTERP_F32):
    """Create a handle for the built-in spline ``name`` (box or Voronoi spline)."""
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(load().interp_create_named(name.encode(), dims.ctypes.data, storage, ctypes.byref(h)),
           "interp_create_named")
    return h


def interp_create(L, xi, dims, storage: int = INTERP_F32):
    """Create a handle for lattice L (s x s) and direction matrix xi (s x n); dims = samples per
    axis of every coset array.  Returns an opaque ctypes pointer."""
    L = np.ascontiguousarray(L, dtype=np.int32)
    xi = np.ascontiguousarray(xi, dtype=np.int32)
    dims = np.ascontiguousarray(dims, dtype=np.int32)
    s = L.shape[0]
    h = ctypes.c_void_p()
    _check(load().interp_create(s, L.ctypes.data, xi.ctypes.data, xi.shape[1], dims.ctypes.data, storage,
                                ctypes.byref(h)), "interp_create")
    return h


def interp_destroy(h):
    if h:
        load().interp_destroy(h)


def interp_info(h) -> InterpInfo:
    info = InterpInfo()
    _check(load().interp_info(h, ctypes.byref(info)), "interp_info")
    return info


def interp_set_option(h, name: str, value: int):
    """Per-handle launch option ("binned", "presort", "dense", "bin_small_tiles"; see the C header)."""
    _check(load().interp_set_option(h, name.encode(), int(value)), "interp_set_option")


def interp_get_option(h, name: str) -> int:
    v = ctypes.c_int()
    _check(load().interp_get_option(h, name.encode(), ctypes.byref(v)), "interp_get_option")
    return v.value


def interp_set_coeffs(h, coeffs, stream=None):
    """coeffs: torch tensor (CUDA or CPU) of float32/float64/float16/bfloat16 in the coset-major
    layout (n_cosets, *dims)."""
    import torch
    dt = {torch.float32: INTERP_F32, torch.float16: INTERP_F16, torch.bfloat16: INTERP_BF16,
          torch.float64: INTERP_F64}[coeffs.dtype]
    c = coeffs.contiguous()
    _check(load().interp_set_coeffs(h, ctypes.c_void_p(c.data_ptr()), dt, int(c.is_cuda),
                                    _stream(stream) if c.is_cuda else _stream(stream)), "interp_set_coeffs")


def interp_prefilter(h, samples, taps, weights, stream=None):
    """coeffs = sum_t w_t samples(n + v_t) (Sec. 5.2's prefilter); samples: CUDA float32 tensor in
    the coefficient layout, taps: (ntaps, s) lattice vectors, weights: (ntaps,)."""
    import torch
    f = _dptr(samples, "samples", torch.float32)
    t = np.ascontiguousarray(taps, dtype=np.int32)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    if t.ndim != 2 or w.shape != (t.shape[0],):
        raise ValueError("taps must be (ntaps, s) and weights (ntaps,)")
    _check(load().interp_prefilter(h, f, t.shape[0], t.ctypes.data, w.ctypes.data, _stream(stream)),
           "interp_prefilter")


def d4_quasi_interpolation_filter():
    """Sec. 5.2's prefilter for the 8-direction spline on D4: 7/3 at the origin and -1/18 at the
    24 lattice vectors of length sqrt(2) (two entries +-1, two zeros).  Returns (taps, weights)."""
    taps = [(0, 0, 0, 0)]
    for a in range(4):
        for b in range(a + 1, 4):
            for sa in (1, -1):
                for sb in (1, -1):
                    v = [0, 0, 0, 0]
                    v[a], v[b] = sa, sb
                    taps.append(tuple(v))
    w = [7.0 / 3.0] + [-1.0 / 18.0] * 24
    return np.asarray(taps, dtype=np.int32), np.asarray(w, dtype=np.float32)


def interp_eval(h, pts, out, stream=None):
    import torch
    _check(load().interp_eval(h, _dptr(pts, "pts", torch.float32), pts.shape[0], _dptr(out, "out", torch.float32),
                              _stream(stream)), "interp_eval")


def interp_eval_grad(h, pts, out, grad, stream=None):
    import torch
    _check(load().interp_eval_grad(h, _dptr(pts, "pts", torch.float32), pts.shape[0],
                                   _dptr(out, "out", torch.float32), _dptr(grad, "grad", torch.float32),
                                   _stream(stream)), "interp_eval_grad")


def interp_eval_host(h, pts, out, grad=None, stream=None):
    """Host (ideally pinned) CPU tensors in and out; copies overlap the evaluation (see the C
    header).  Synchronise the stream before reading out / grad."""
    import torch
    for t, nm in ((pts, "pts"), (out, "out"), (grad, "grad")):
        if t is not None and (t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous()):
            raise ValueError(f"{nm} must be a contiguous float32 CPU tensor")
    _check(load().interp_eval_host(h, ctypes.c_void_p(pts.data_ptr()), pts.shape[0], ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(grad.data_ptr()) if grad is not None else None, _stream(stream)),
           "interp_eval_host")


def interp_sort_points(h, pts, perm=None, pts_sorted=None, stream=None):
    """Spatial counting sort of the queries (see the C header); fills perm (int32) and/or
    pts_sorted."""
    import torch
    _check(load().interp_sort_points(h, _dptr(pts, "pts", torch.float32), pts.shape[0],
                                     _dptr(perm, "perm", torch.int32), _dptr(pts_sorted, "pts_sorted", torch.float32),
                                     _stream(stream)), "interp_sort_points")


def interp_backward(h, pts, gout, dcoeffs, dpts=None, stream=None):
    import torch
    _check(load().interp_backward(h, _dptr(pts, "pts", torch.float32), pts.shape[0],
                                  _dptr(gout, "gout", torch.float32), _dptr(dcoeffs, "dcoeffs", torch.float32),
                                  _dptr(dpts, "dpts", torch.float32), _stream(stream)), "interp_backward")


def interp_backward_noalloc(h, pts, gout, dcoeffs, dpts=None, stream=None):
    """The adjoint without any device allocation (scratch in a static device array); see the C
    header for its size limit and the rule that overlapping calls race."""
    import torch
    _check(load().interp_backward_noalloc(h, _dptr(pts, "pts", torch.float32), pts.shape[0],
                                          _dptr(gout, "gout", torch.float32),
                                          _dptr(dcoeffs, "dcoeffs", torch.float32),
                                          _dptr(dpts, "dpts", torch.float32), _stream(stream)),
           "interp_backward_noalloc")


def interp_debug_indices(h, pts, cells=None, piece=None, stream=None):
    import torch
    _check(load().interp_debug_indices(h, _dptr(pts, "pts", torch.float32), pts.shape[0],
                                       _dptr(cells, "cells", torch.int32), _dptr(piece, "piece", torch.int32),
                                       _stream(stream)), "interp_debug_indices")


def make_rays(origin, du, dv, direction, box_lo, box_hi, width, height, steps) -> Rays:
    r = Rays()
    for name, v in (("origin", origin), ("du", du), ("dv", dv), ("dir", direction), ("box_lo", box_lo),
                    ("box_hi", box_hi)):
        getattr(r, name)[:] = [float(a) for a in v]
    r.width, r.height, r.steps = int(width), int(height), int(steps)
    return r


def interp_eval_rays(h, rays: Rays, out, with_grad: bool = False, pts_out=None, stream=None):
    """Per-pixel sums of f (and grad f) along orthographic rays; see the C header."""
    import torch
    _check(load().interp_eval_rays(h, ctypes.byref(rays), int(with_grad), _dptr(out, "out", torch.float32),
                                   _dptr(pts_out, "pts_out", torch.float32), _stream(stream)), "interp_eval_rays")


def interp_batch_create(items):
    """items: list of (handle, pts tensor, out tensor).  The tensors must outlive the batch."""
    import torch
    arr = (BatchItem * len(items))()
    for i, (h, pts, out) in enumerate(items):
        arr[i].vol = h.value if isinstance(h, ctypes.c_void_p) else h
        arr[i].pts = _dptr(pts, "pts", torch.float32).value if pts.numel() else None
        arr[i].npts = pts.shape[0]
        arr[i].out = _dptr(out, "out", torch.float32).value if out.numel() else None
    b = ctypes.c_void_p()
    _check(load().interp_batch_create(arr, len(items), ctypes.byref(b)), "interp_batch_create")
    return b


def interp_batch_autotune(b, stream=None):
    _check(load().interp_batch_autotune(b, _stream(stream)), "interp_batch_autotune")


def interp_batch_tile(b, spline: str) -> int:
    t = ctypes.c_int()
    _check(load().interp_batch_tile(b, spline.encode(), ctypes.byref(t)), "interp_batch_tile")
    return t.value


def interp_batch_set_tile(b, spline: str, tile: int):
    _check(load().interp_batch_set_tile(b, spline.encode(), tile), "interp_batch_set_tile")


def interp_batch_run(b, stream=None):
    _check(load().interp_batch_run(b, _stream(stream)), "interp_batch_run")


def interp_batch_destroy(b):
    if b:
        load().interp_batch_destroy(b)


class Batch:
    """Many (Interpolator, points, output) triples evaluated by one persistent launch (plus one
    launch per handle outside the persistent kernel's splines), replayed from a CUDA graph."""

    def __init__(self, items):
        self._keep = list(items)        # keep the handles and tensors alive
        self._b = interp_batch_create([(it.handle, p, o) for it, p, o in items])

    def autotune(self, stream=None) -> dict:
        interp_batch_autotune(self._b, stream)
        return self.tiles()

    def tiles(self) -> dict:
        """Tile size per spline of the persistent kernel (handles that run their own launch, the
        4-D ones and the 3-D splines outside the persistent kernel, have none)."""
        out = {}
        for n in sorted({it.info.name.decode() for it, _, _ in self._keep if it.s == 3}):
            try:
                out[n] = interp_batch_tile(self._b, n)
            except InterpError:
                pass
        return out

    def set_tiles(self, tiles: dict):
        for n, t in tiles.items():
            interp_batch_set_tile(self._b, n, t)

    def run(self, stream=None):
        interp_batch_run(self._b, stream)

    def close(self):
        if getattr(self, "_b", None):
            interp_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- convenience object

STORAGE = {"f32": INTERP_F32, "f16": INTERP_F16, "bf16": INTERP_BF16}


class Interpolator:
    """A handle plus its shape: f(x) = sum_k sum_i c_k[i] phi(x - D i - l_k) on one device.

    Interpolator(L, xi, dims) selects a box spline by lattice and direction matrix;
    Interpolator.named(name, dims) any built-in spline by name (the Voronoi splines have no
    direction matrix)."""

    def __init__(self, L, xi, dims, storage: str = "f32", coeffs=None, *, name: str | None = None):
        self.dims = tuple(int(d) for d in dims)
        self.storage = storage
        if name is not None:
            self._h = interp_create_named(name, self.dims, STORAGE[storage])
            self.L = self.xi = None
        else:
            self.L = np.asarray(L, dtype=np.int32)
            self.xi = np.asarray(xi, dtype=np.int32)
            self._h = interp_create(self.L, self.xi, self.dims, STORAGE[storage])
        self.info = interp_info(self._h)
        self.s = self.info.s
        self.n_cosets = self.info.n_cosets
        self.shape = (self.n_cosets,) + self.dims
        if coeffs is not None:
            self.set_coeffs(coeffs)

    @classmethod
    def named(cls, name: str, dims, storage: str = "f32", coeffs=None):
        return cls(None, None, dims, storage, coeffs, name=name)

    def close(self):
        if getattr(self, "_h", None):
            interp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_coeffs(self, coeffs, stream=None):
        if tuple(coeffs.shape) != self.shape:
            raise ValueError(f"coefficients must have shape {self.shape}, got {tuple(coeffs.shape)}")
        interp_set_coeffs(self._h, coeffs, stream)

    def set_option(self, name: str, value: int):
        interp_set_option(self._h, name, value)

    def get_option(self, name: str) -> int:
        return interp_get_option(self._h, name)

    def prefilter(self, samples, taps, weights, stream=None):
        """Coefficients from samples by a lattice filter (interp_prefilter)."""
        if tuple(samples.shape) != self.shape:
            raise ValueError(f"samples must have shape {self.shape}, got {tuple(samples.shape)}")
        interp_prefilter(self._h, samples, taps, weights, stream)

    def eval(self, pts, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(pts.shape[0], device=pts.device, dtype=torch.float32)
        interp_eval(self._h, pts, out, stream)
        return out

    def eval_grad(self, pts, out=None, grad=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(pts.shape[0], device=pts.device, dtype=torch.float32)
        if grad is None:
            grad = torch.empty(pts.shape[0], self.s, device=pts.device, dtype=torch.float32)
        interp_eval_grad(self._h, pts, out, grad, stream)
        return out, grad

    def backward(self, pts, gout, dcoeffs=None, want_dpts=False, stream=None):
        import torch
        if dcoeffs is None:
            dcoeffs = torch.zeros(self.shape, device=pts.device, dtype=torch.float32)
        dpts = torch.empty(pts.shape[0], self.s, device=pts.device, dtype=torch.float32) if want_dpts else None
        interp_backward(self._h, pts, gout, dcoeffs, dpts, stream)
        return dcoeffs, dpts

    def sort_points(self, pts, stream=None):
        """(permutation, sorted points): queries reordered so that neighbours in space are
        neighbours in memory."""
        import torch
        perm = torch.empty(pts.shape[0], device=pts.device, dtype=torch.int32)
        out = torch.empty_like(pts)
        interp_sort_points(self._h, pts, perm, out, stream)
        return perm, out

    def debug_indices(self, pts, stream=None):
        import torch
        cells = torch.empty(pts.shape[0], self.n_cosets, self.s, device=pts.device, dtype=torch.int32)
        piece = torch.empty(pts.shape[0], self.n_cosets, device=pts.device, dtype=torch.int32)
        interp_debug_indices(self._h, pts, cells, piece, stream)
        return cells, piece


def _autograd_function():
    import torch

    class LatticeInterp(torch.autograd.Function):
        """f = LatticeInterp.apply(pts, coeffs, interpolator): forward runs interp_eval with the
        handle's coefficients set from `coeffs`; backward runs the hand-written adjoint
        (dL/dcoeffs by the scatter kernel, dL/dpts = g * grad f)."""

        @staticmethod
        def forward(ctx, pts, coeffs, interp: Interpolator):
            interp.set_coeffs(coeffs.detach())
            ctx.interp = interp
            ctx.save_for_backward(pts)
            return interp.eval(pts.detach().contiguous())

        @staticmethod
        def backward(ctx, g):
            (pts,) = ctx.saved_tensors
            interp = ctx.interp
            want_c = ctx.needs_input_grad[1]
            want_x = ctx.needs_input_grad[0]
            dc = torch.zeros(interp.shape, device=pts.device, dtype=torch.float32) if want_c else None
            dx = torch.empty(pts.shape[0], interp.s, device=pts.device, dtype=torch.float32) if want_x else None
            interp_backward(interp.handle, pts.detach().contiguous(), g.contiguous().float(), dc, dx)
            return dx, dc, None

    return LatticeInterp


_LatticeInterp = None


def lattice_interp(pts, coeffs, interp: Interpolator):
    """Differentiable f(pts) w.r.t. pts and coeffs (autograd through the hand-written adjoint)."""
    global _LatticeInterp
    if _LatticeInterp is None:
        _LatticeInterp = _autograd_function()
    return _LatticeInterp.apply(pts, coeffs, interp)
