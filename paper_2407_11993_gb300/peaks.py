"""Measured arithmetic peaks of the current GPU (roofline denominators).

``measure()`` runs register-resident multiply-add loops over every SM -- FP64 FMA on
the CUDA cores, FP64 ``mma.sync`` (m8n8k4) on the tensor path, FP32 FMA -- and returns
the best of ``reps`` event-timed launches in TFLOP/s.  HBM bandwidth and BF16 GEMM
peaks come from the pool's own measurement file; these cover the FP64 / FP32 pipes
that the FP64 eddy-current kernels are bound by.

    python -m paper_2407_11993_gb300.peaks        # prints one JSON line
"""
from __future__ import annotations

import ctypes
import json


def measure(reps: int = 5) -> dict:
    from paper_2407_11993_gb300 import build
    path = build.build_peaks()
    lib = ctypes.CDLL(path)
    lib.ec_peak_probe.restype = ctypes.c_int
    lib.ec_peak_probe.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = (ctypes.c_double * 6)()
    rc = lib.ec_peak_probe(int(reps), out)
    if rc != 0:
        raise RuntimeError(f"peak probe failed with CUDA error {rc}")
    return {"fp64_fma_tflops": out[0], "fp64_mma_tflops": out[1], "fp32_fma_tflops": out[2],
            "sms": int(out[3]), "sm_clock_mhz_reported": out[4],
            "fp64_fma_and_mma_together_tflops": out[5], "reps": int(reps)}


if __name__ == "__main__":
    print(json.dumps(measure()))
