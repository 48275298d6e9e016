"""Measured throughput of the FP64 pipe and of the integer pipe on the
current GPU (``_build/libqp_peaks.so``, built from ``csrc/peaks.cu``).

The EN-PT2 sweep is gather-and-bit work with FP64 arithmetic: neither HBM
nor the tensor cores bound it.  Its roofline is therefore reported against
these two measured rates: FP64 FMAs per second, and integer XOR / POPC / add
operations per second (the excitation-degree tests and phases).
"""
from __future__ import annotations

import ctypes as C
import os

from .build import PEAKS_SO

_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(PEAKS_SO):
            raise ImportError(f"peaks library not built: {PEAKS_SO}")
        _lib = C.CDLL(PEAKS_SO)
        _lib.qp_peak_measure.restype = C.c_int
        _lib.qp_peak_measure.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]
    return _lib


def measure(kind: str, iters: int = 4096, reps: int = 6) -> dict:
    """kind 'fp64' (FMA) or 'int' (XOR/POPC/add).  Best of reps after a
    warm-up; returns G operations per second, operations per SM clock, the
    kernel time and the SM clock implied by clock64."""
    out = (C.c_double * 4)()
    rc = _load().qp_peak_measure(0 if kind == "fp64" else 1, int(iters), int(reps), out)
    if rc != 0:
        raise RuntimeError(f"peak measurement failed (code {rc})")
    return {"gops": out[0], "ops_per_sm_clock": out[1], "ms": out[2], "implied_sm_mhz": out[3]}
