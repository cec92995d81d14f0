"""The measured-peaks microbenchmarks that check a result: the tensor-core TF32 product
(tcgen05.mma kind::tf32 with shared-memory operands in the 128-byte swizzle and the accumulator
in TMEM) against the host, with inputs that TF32 holds exactly, so the comparison is exact."""
import ctypes

import pytest

from _gpu_common import require_cuda

pytestmark = pytest.mark.gpu


def test_tensor_core_tf32_product_is_exact():
    torch = require_cuda()
    from paper_2102_08514_b300 import peaks
    lib = ctypes.CDLL(peaks.library_path())
    lib.peaks_tc_tf32.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.peaks_tc_tf32.restype = ctypes.c_int
    g = torch.Generator().manual_seed(7)
    for scale in (4, 16):
        a = (torch.randint(-scale, scale + 1, (128, 32), generator=g).float() / scale).cuda()
        b = (torch.randint(-scale, scale + 1, (128, 32), generator=g).float() / scale).cuda()
        d = torch.full((128, 128), float("nan"), device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert lib.peaks_tc_tf32(a.data_ptr(), b.data_ptr(), d.data_ptr(), 1, 1, err.data_ptr(), None) == 0
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert torch.equal(d, (a.double() @ b.double().T).float())
