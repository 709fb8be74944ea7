"""Measured hardware rates of the current GPU (the roofline denominators).

Runs the library's microbenchmarks (``rt_peak_fma``, ``rt_peak_gather``,
``rt_peak_read``; include/rt.h) on the current device and stream and times
each launch with CUDA events: FP32 and FP64 fused multiply-add rates, random
16-byte gathers from a 16 MiB L2-resident buffer, and coalesced reads of a
32 MiB L2-resident buffer. Each figure is the best of ``reps`` launches after
one warm-up launch.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as _L

THREADS = 256


def _sms() -> int:
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _best_ms(launch, reps: int) -> float:
    s = torch.cuda.current_stream()
    launch()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        launch()
        b.record(s)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def measure(reps: int = 5) -> dict:
    """Rates of the current device: FP32/FP64 TFLOP/s, L2 gather and read GB/s."""
    lib = _L.load()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    sms = _sms()
    blocks = sms * 8                      # 2048 resident threads per SM
    n = blocks * THREADS
    sink32 = torch.empty(n, dtype=torch.float32, device="cuda")
    sink64 = torch.empty(n, dtype=torch.float64, device="cuda")

    def fma(dtype, iters):
        sink = sink32 if dtype == 0 else sink64
        return lambda: _L.check(None, lib.rt_peak_fma(dtype, blocks, iters, C.c_void_p(sink.data_ptr()), s))

    it32, it64 = 16384, 512
    ms32 = _best_ms(fma(0, it32), reps)
    ms64 = _best_ms(fma(1, it64), reps)
    fp32 = blocks * THREADS * it32 * 16 / (ms32 * 1e-3) / 1e12
    fp64 = blocks * THREADS * it64 * 16 / (ms64 * 1e-3) / 1e12

    n_vec = 1 << 20                       # 16 MiB of float4
    buf = torch.rand(n_vec * 4, dtype=torch.float32, device="cuda")
    g_iters = 256
    msg = _best_ms(lambda: _L.check(None, lib.rt_peak_gather(C.c_void_p(buf.data_ptr()), n_vec, blocks, g_iters,
                                                              C.c_void_p(sink32.data_ptr()), s)), reps)
    gather = blocks * THREADS * g_iters * 128 / (msg * 1e-3) / 1e9

    n_read = 1 << 21                      # 32 MiB of float4
    buf2 = torch.rand(n_read * 4, dtype=torch.float32, device="cuda")
    passes = 64
    msr = _best_ms(lambda: _L.check(None, lib.rt_peak_read(C.c_void_p(buf2.data_ptr()), n_read, blocks, passes,
                                                            C.c_void_p(sink32.data_ptr()), s)), reps)
    read = passes * n_read * 16 / (msr * 1e-3) / 1e9
    return {"fp32_tflops": fp32, "fp64_tflops": fp64, "l2_gather_gbs": gather, "l2_read_gbs": read,
            "sms": sms, "how": ("rt_peak_fma (8 FMA chains per thread, 2048 threads per SM), rt_peak_gather "
                                "(random float4 from 16 MiB), rt_peak_read (coalesced float4 over 32 MiB, 64 "
                                f"passes); best of {reps} launches, CUDA events")}
