"""Measured arithmetic peaks of the current GPU (ctypes binding of
``libharm_peaks.so``, include/harm_peaks.h): FP32 FMA, packed FP32x2 FMA, FP64
FMA (TFLOP/s) and __sinf evaluations (per clock per SM at the sampled clock is
left to the caller). Each figure is the best of a few CUDA-event-timed launches."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libharm_peaks.so")
KINDS = {"ffma": 0, "ffma2": 1, "dfma": 2, "sinf": 3}
_lib = None


def load_library(path: str = LIB_PATH):
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libharm_peaks.so not built at %s" % path)
        lib = C.CDLL(path)
        lib.harm_peak_launch.restype = C.c_int
        lib.harm_peak_launch.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        lib.harm_peak_ops.restype = C.c_longlong
        lib.harm_peak_ops.argtypes = [C.c_int, C.c_int, C.c_int]
        _lib = lib
    return _lib


# iterations per launch: ~1 ms (FP32), ~10 ms (FP64, __sinf) on a B300
ITERS = {"ffma": 16384, "ffma2": 8192, "dfma": 2048, "sinf": 8192}


def measure(kind: str, iters: int = 0, repeats: int = 5, ctas_per_sm: int = 8):
    """Rate of benchmark `kind` on the current device: (operations per second,
    best launch in ms, SM count), best of `repeats` launches after one warm-up."""
    import torch
    lib = load_library()
    iters = iters or ITERS[kind]
    k = KINDS[kind]
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * ctas_per_sm
    out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    best = None
    for i in range(repeats + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rc = lib.harm_peak_launch(k, blocks, iters, C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        b.record(stream)
        if rc != 0:
            raise RuntimeError("harm_peak_launch(%s) failed: %d" % (kind, rc))
        torch.cuda.synchronize()
        if i > 0:
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
    ops = lib.harm_peak_ops(k, blocks, iters)
    return ops / (best * 1e-3), best, sms
