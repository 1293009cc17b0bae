"""The FP32 FMA probe behind the roofline denominator: FLOP count and a plausible rate."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fma_probe_rate():
    from paper_2508_17187_gb300 import _lib
    lib = _lib.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n_blocks, iters = sms * 8, 1 << 16
    out = torch.empty(n_blocks * 256, dtype=torch.float32, device="cuda")
    flop = ctypes.c_double()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    assert lib.awg_fp32_fma_probe(ctypes.c_void_p(out.data_ptr()), n_blocks, iters, sp, ctypes.byref(flop)) == 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    assert lib.awg_fp32_fma_probe(ctypes.c_void_p(out.data_ptr()), n_blocks, iters, sp, ctypes.byref(flop)) == 0
    e1.record(stream)
    torch.cuda.synchronize()
    assert flop.value == 2 * 8 * iters * n_blocks * 256
    assert torch.isfinite(out).all()
    tflops = flop.value / (e0.elapsed_time(e1) / 1e3) / 1e12
    # 128 FP32 lanes per SM at 0.5-2.5 GHz
    assert sms * 128 * 2 * 0.5e9 / 1e12 < tflops < sms * 128 * 2 * 2.5e9 / 1e12, tflops
    assert lib.awg_fp32_fma_probe(ctypes.c_void_p(out.data_ptr()), 0, iters, sp, ctypes.byref(flop)) == 1


def test_fp64_fma_probe_rate():
    """The FP64 probe: FLOP count, finite output and a rate between 1/128 and 1/2 of the FP32 lanes'
    (GB300's FP64 pipe is a small fraction of its FP32 pipe)."""
    from paper_2508_17187_gb300 import _lib
    lib = _lib.load()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n_blocks, iters = sms * 8, 1 << 10
    out = torch.empty(n_blocks * 256, dtype=torch.float64, device="cuda")
    flop = ctypes.c_double()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    assert lib.awg_fp64_fma_probe(ctypes.c_void_p(out.data_ptr()), n_blocks, iters, sp, ctypes.byref(flop)) == 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    assert lib.awg_fp64_fma_probe(ctypes.c_void_p(out.data_ptr()), n_blocks, iters, sp, ctypes.byref(flop)) == 0
    e1.record(stream)
    torch.cuda.synchronize()
    assert flop.value == 2 * 8 * iters * n_blocks * 256
    assert torch.isfinite(out).all()
    tflops = flop.value / (e0.elapsed_time(e1) / 1e3) / 1e12
    fp32_max = sms * 128 * 2 * 2.5e9 / 1e12
    assert fp32_max / 256 < tflops < fp32_max / 2, tflops
