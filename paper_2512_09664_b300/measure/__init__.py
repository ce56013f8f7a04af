"""ALU throughput probes for the benchmark's roofline (``libsynthpix_probe.so``).

Measurement support only: the probes time FP32 FMA, ``erfcf``, the SFU
exponential and the Philox high multiply on the current device.  They are no
part of the renderer or of its C ABI.  Raises if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB_PATH = os.path.join(_PKG, "libsynthpix_probe.so")
KINDS = {"fma": 0, "erfc": 1, "ex2": 2, "umulhi": 3}
EINVAL, ECUDA = -1, -3
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2512_09664_b300.build`")
        L = C.CDLL(LIB_PATH)
        L.synthpix_alu_probe_threads.argtypes = []
        L.synthpix_alu_probe_threads.restype = C.c_int64
        L.synthpix_alu_probe.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.POINTER(C.c_int64),
                                         C.c_void_p]
        L.synthpix_alu_probe.restype = C.c_int
        L.synthpix_probe_last_error.argtypes = []
        L.synthpix_probe_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def last_error() -> str:
    return lib().synthpix_probe_last_error().decode()


def alu_probe(kind: str, iters: int = 4096, reps: int = 3, stream=None) -> float:
    """Best of `reps` timed synthpix_alu_probe launches: operations per second.

    kind is one of KINDS; the launches run on `stream` (default: the current
    one) and are timed with CUDA events there (this synchronises).
    """
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    n = lib().synthpix_alu_probe_threads()
    if n <= 0:
        raise RuntimeError(f"alu probe: {last_error()}")
    sink = torch.empty(n, dtype=torch.float32, device=st.device)
    ops = C.c_int64(0)
    best = 0.0
    for _ in range(reps + 1):  # the first launch is a warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc = lib().synthpix_alu_probe(KINDS[kind], iters, C.c_void_p(sink.data_ptr()), n, C.byref(ops),
                                      C.c_void_p(st.cuda_stream))
        if rc != 0:
            raise RuntimeError(f"alu probe error {rc}: {last_error()}")
        e1.record(st)
        e1.synchronize()
        best = max(best, ops.value / (e0.elapsed_time(e1) * 1e-3))
    return best
