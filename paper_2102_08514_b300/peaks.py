"""Measured peaks of the resources the evaluator is bound by (one GPU).

    python -m paper_2102_08514_b300.peaks            # prints one JSON line

`measure()` runs the microbenchmarks of `csrc/peaks.cu` on the current CUDA device and stream
(CUDA events, warm-up, best of several launches) and returns:

* ``fp32_tflops`` -- FP32 FMA throughput (2 FLOP per FMA), the roofline of work whose gathers
  hit L1 (ray-coherent or spatially sorted queries);
* ``l2_read_gbs`` -- coalesced reads of a buffer that fits L2;
* ``gather_gsectors_s`` -- scalar 4-byte loads at pseudo-random addresses of an L2-resident
  buffer, one 32-byte sector (one L1 -> L2 miss request) each: the rate that bounds the
  coefficient gathers of random queries; ``gather{4,16,32}B_{l2,l1}_gloads_s`` the same for
  4-, 16- and 32-byte loads from L2- and L1-resident buffers (L1 lookups of divergent loads);
* ``gather_line{1,2,4}_gsectors_s`` -- the same 4-byte gathers with groups of 1, 2 or 4 lanes
  reading different sectors of one pseudo-random 128-byte line in every instruction: sectors per
  second when one L1 -> L2 request carries 1, 2 or 4 sectors;
* ``tc_tf32_tflops`` -- tensor-core TF32 products by ``tcgen05.mma kind::tf32`` (one CTA per SM,
  operands in shared memory, accumulator in TMEM); ``tc_tf32_product_exact`` -- one 128 x 128 x 32
  product with TF32-exact inputs equals the host's;
* ``red_gatomics_s`` -- red.global.add.f32 at pseudo-random addresses of an L2-resident buffer
  (the adjoint's scatter);
* ``shared_atomic_{f32,u32,u64}_gops_s`` -- shared-memory atomic adds at pseudo-random elements:
  float, 32- and 64-bit integer (the binned adjoint's per-bin sums); ``shared_fixed64_gops_s``
  a 64-bit fixed-point add kept as two 32-bit words (low word with carry out).

The SM count comes from the device; the caller samples the SM clock around the calls (the
per-clock figures divide by it).
"""
from __future__ import annotations

import ctypes
import json
import os

_LIB = None


def library_path() -> str:
    from . import build
    return build.build_peaks()


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(library_path())
        v = ctypes.c_void_p
        _LIB.peaks_fma.argtypes = [ctypes.c_int, ctypes.c_int, v, v]
        _LIB.peaks_l2_read.argtypes = [v, ctypes.c_int64, ctypes.c_int, ctypes.c_int, v, v]
        _LIB.peaks_gather.argtypes = [v, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int, v, v]
        _LIB.peaks_gather_lines.argtypes = [v, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int, v, v]
        _LIB.peaks_red.argtypes = [v, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, v]
        _LIB.peaks_tc_tf32.argtypes = [v, v, v, ctypes.c_int, ctypes.c_int, v, v]
        _LIB.peaks_shared_atomic.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, v, v]
        for f in (_LIB.peaks_fma, _LIB.peaks_l2_read, _LIB.peaks_gather, _LIB.peaks_gather_lines, _LIB.peaks_red,
                  _LIB.peaks_shared_atomic, _LIB.peaks_tc_tf32):
            f.restype = ctypes.c_int
    return _LIB


def _best_ms(torch, launch, reps: int = 5, warm: int = 2) -> float:
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        launch()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        launch()
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what}: CUDA error {rc}")


def measure(torch=None) -> dict:
    """Run the microbenchmarks on the current device; rates as documented above."""
    if torch is None:
        import torch
    lib = _lib()
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    res = {"sms": sms}

    # FP32 FMA: 8 CTAs of 256 threads per SM (full occupancy)
    grid, iters = sms * 8, 600
    scratch = torch.empty(grid * 256, device="cuda")
    ms = _best_ms(torch, lambda: _check(lib.peaks_fma(grid, iters, ctypes.c_void_p(scratch.data_ptr()), st),
                                        "peaks_fma"))
    res["fp32_tflops"] = grid * 256 * 8 * 64 * iters * 2 / (ms * 1e-3) / 1e12
    res["fp32_ms"] = ms

    # L2-resident read: 32 MiB read 64 times
    n4 = (32 << 20) // 16
    buf = torch.ones(n4 * 4, device="cuda")
    passes = 64
    ms = _best_ms(torch, lambda: _check(lib.peaks_l2_read(ctypes.c_void_p(buf.data_ptr()), n4, passes, grid,
                                                          ctypes.c_void_p(scratch.data_ptr()), st), "peaks_l2_read"))
    res["l2_read_gbs"] = n4 * 16 * passes / (ms * 1e-3) / 1e9
    res["l2_read_bytes"] = n4 * 16

    # random gathers: 16 CTAs of 128 threads per SM, 8 independent loads per thread and round,
    # from 16 MiB (L2-resident, the size of a bricked coefficient array) and from 32 KiB
    # (L1-resident), of 4, 16 and 32 bytes
    words = 1 << 22
    gbuf = torch.ones(words, device="cuda")
    ggrid, giters = sms * 16, 128
    gout = torch.empty(ggrid * 128, device="cuda")
    loads = ggrid * 128 * 8 * giters
    for where, nbytes in (("l2", words * 4), ("l1", 32 << 10)):
        for width in (1, 4, 8):
            mask = nbytes // (4 * width) - 1
            ms = _best_ms(torch, lambda: _check(lib.peaks_gather(ctypes.c_void_p(gbuf.data_ptr()), mask, width, ggrid,
                                                                 giters, ctypes.c_void_p(gout.data_ptr()), st),
                                                "peaks_gather"))
            res[f"gather{width * 4}B_{where}_gloads_s"] = loads / (ms * 1e-3) / 1e9
    res["gather_gsectors_s"] = res["gather4B_l2_gloads_s"]
    res["gather_buffer_bytes"] = words * 4
    # the same 16 MiB as lines of 128 bytes, 1, 2 or 4 lanes per line and instruction
    for group in (1, 2, 4):
        ms = _best_ms(torch, lambda: _check(lib.peaks_gather_lines(ctypes.c_void_p(gbuf.data_ptr()), words // 32 - 1,
                                                                   group, ggrid, giters,
                                                                   ctypes.c_void_p(gout.data_ptr()), st),
                                            "peaks_gather_lines"))
        res[f"gather_line{group}_gsectors_s"] = loads / (ms * 1e-3) / 1e9

    # random L2 atomics into 16 MiB
    rbuf = torch.zeros(words, device="cuda")
    riters = 64
    ms = _best_ms(torch, lambda: _check(lib.peaks_red(ctypes.c_void_p(rbuf.data_ptr()), words - 1, ggrid, riters, st),
                                        "peaks_red"))
    res["red_gatomics_s"] = ggrid * 128 * 4 * riters / (ms * 1e-3) / 1e9

    # shared-memory atomics, float and integer add: 8 CTAs of 256 threads per SM
    sgrid, siters = sms * 8, 64
    sout = torch.empty(sgrid, device="cuda")
    for t, name in ((0, "shared_atomic_f32_gops_s"), (1, "shared_atomic_u32_gops_s"), (2, "shared_atomic_u64_gops_s"),
                    (3, "shared_fixed64_gops_s")):
        ms = _best_ms(torch, lambda: _check(lib.peaks_shared_atomic(t, sgrid, siters, ctypes.c_void_p(sout.data_ptr()), st),
                                            "peaks_shared_atomic"))
        res[name] = sgrid * 256 * 8 * siters / (ms * 1e-3) / 1e9
    # tensor cores (tcgen05.mma kind::tf32): one exact 128 x 128 x 32 product checked against the
    # host (inputs that TF32 holds exactly), then the rate of accumulating products
    g = torch.Generator().manual_seed(2102)
    ta = (torch.randint(-4, 5, (128, 32), generator=g).float() / 4).cuda()
    tb = (torch.randint(-4, 5, (128, 32), generator=g).float() / 4).cuda()
    td = torch.full((128, 128), float("nan"), device="cuda")
    terr = torch.zeros(1, dtype=torch.int32, device="cuda")
    _check(lib.peaks_tc_tf32(ctypes.c_void_p(ta.data_ptr()), ctypes.c_void_p(tb.data_ptr()),
                             ctypes.c_void_p(td.data_ptr()), 1, 1, ctypes.c_void_p(terr.data_ptr()), st),
           "peaks_tc_tf32")
    torch.cuda.synchronize()
    ref = (ta.double() @ tb.double().T).float()
    res["tc_tf32_product_exact"] = bool(int(terr.item()) == 0 and torch.equal(td, ref))
    tgrid, titers = sms, 2048
    ms = _best_ms(torch, lambda: _check(lib.peaks_tc_tf32(ctypes.c_void_p(ta.data_ptr()), ctypes.c_void_p(tb.data_ptr()),
                                                          ctypes.c_void_p(td.data_ptr()), tgrid, titers,
                                                          ctypes.c_void_p(terr.data_ptr()), st), "peaks_tc_tf32"))
    res["tc_tf32_tflops"] = tgrid * titers * 2.0 * 128 * 128 * 32 / (ms * 1e-3) / 1e12
    res["tc_tf32_timeouts"] = int(terr.item())
    torch.cuda.synchronize()
    return res


def per_clock(res: dict, sm_mhz: float) -> dict:
    """The rates per SM and SM clock cycle at the sampled clock."""
    hz = sm_mhz * 1e6
    sms = res["sms"]
    return {"fp32_flop_per_clk_per_sm": res["fp32_tflops"] * 1e12 / (sms * hz),
            "l2_read_bytes_per_clk_per_sm": res["l2_read_gbs"] * 1e9 / (sms * hz),
            "gather_sectors_per_clk_per_sm": res["gather_gsectors_s"] * 1e9 / (sms * hz),
            **{k.replace("_gloads_s", "_loads_per_clk_per_sm"): v * 1e9 / (sms * hz)
               for k, v in res.items() if k.endswith("_gloads_s")},
            "red_per_clk_per_sm": res["red_gatomics_s"] * 1e9 / (sms * hz),
            "shared_atomic_f32_per_clk_per_sm": res["shared_atomic_f32_gops_s"] * 1e9 / (sms * hz),
            "shared_atomic_u32_per_clk_per_sm": res["shared_atomic_u32_gops_s"] * 1e9 / (sms * hz),
            "shared_atomic_u64_per_clk_per_sm": res["shared_atomic_u64_gops_s"] * 1e9 / (sms * hz)}


if __name__ == "__main__":
    import torch
    print(json.dumps(measure(torch)))
