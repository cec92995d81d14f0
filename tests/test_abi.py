"""The C-ABI library builds, loads and exports every entry point include/interp.h declares; the
argument checks that need no GPU behave as documented (no kernel launches here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2102_08514_b300 import build as b
    path = b.build()
    return ctypes.CDLL(path), path


def declared_functions():
    text = open(os.path.join(ROOT, "include", "interp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(interp_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    handle, path = lib
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(handle, n), n
    from paper_2102_08514_b300.binding import exported_symbols
    assert sorted(exported_symbols()) == names


def test_registry_and_strerror(lib):
    from paper_2102_08514_b300 import binding
    binding.load(lib[1])
    names = binding.spline_names()
    assert set(names) >= {"bcc_linear", "bcc_quintic", "fcc_6dir", "cc_7dir", "d4s_8dir"}
    assert len(binding.table_digest()) == 16
    for st in range(6):
        assert binding._strerror(st)


def test_create_argument_errors_without_gpu(lib):
    # these are rejected before any CUDA call
    from paper_2102_08514_b300 import binding
    from synth import LATTICES, SPLINES
    L = np.asarray(LATTICES["bcc"].L)
    xi = np.asarray(SPLINES["bcc_quintic"].xi)
    with pytest.raises(binding.InterpError) as e:
        binding.interp_create(np.zeros((3, 3)), xi, (8, 8, 8))
    assert e.value.status == binding.INTERP_EINVAL
    with pytest.raises(binding.InterpError) as e:
        binding.interp_create(L, xi[:, :6], (8, 8, 8))
    assert e.value.status == binding.INTERP_EUNSUPPORTED
    with pytest.raises(binding.InterpError) as e:
        binding.interp_create(L, xi, (8, 0, 8))
    assert e.value.status == binding.INTERP_EINVAL
    with pytest.raises(binding.InterpError) as e:
        binding.interp_create(np.eye(2, dtype=int), np.eye(2, dtype=int), (8, 8))
    assert e.value.status == binding.INTERP_EUNSUPPORTED
    # padded FP32 arrays of 2 x 1024^3 elements (dims 1015^3 + halo, rounded to whole bricks)
    # exceed the 32-bit element offsets: refused before any allocation (1014^3 fits, GPU test)
    with pytest.raises(binding.InterpError) as e:
        binding.interp_create(L, xi, (1015, 1015, 1015))
    assert e.value.status == binding.INTERP_ESIZE
    h = binding.load()
    assert h.interp_eval(None, None, 0, None, None) == binding.INTERP_EINVAL


def test_option_argument_errors_without_gpu(lib):
    from paper_2102_08514_b300 import binding
    h = binding.load()
    assert h.interp_set_option(None, b"binned", 1) == binding.INTERP_EINVAL
    v = ctypes.c_int()
    assert h.interp_get_option(None, b"presort", ctypes.byref(v)) == binding.INTERP_EINVAL
    assert h.interp_debug_device_allocations() >= 0


def test_peaks_library_exports_its_microbenchmarks():
    import ctypes
    from paper_2102_08514_b300 import peaks
    plib = ctypes.CDLL(peaks.library_path())
    for name in ("peaks_fma", "peaks_l2_read", "peaks_gather", "peaks_gather_lines", "peaks_red", "peaks_tc_tf32",
                 "peaks_shared_atomic"):
        assert hasattr(plib, name), name
