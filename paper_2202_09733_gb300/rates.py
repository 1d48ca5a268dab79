"""Arithmetic rates of this GPU's FP64 and FP32 pipes (csrc/rates.cu): scalar FP64 fma
chains (DFMA), the FP64 tensor-core MMA (DMMA, m8n8k4) and scalar FP32 fma chains, each
timed with CUDA events over one launch of 8 CTAs of 256 threads per SM.

    python -m paper_2202_09733_gb300.rates [--iters N]

prints one JSON line {"dfma_tflops", "dmma_tflops", "ffma_tflops"}.  These rates decide
where the FP64 residual's operator applications run (DFMA chains in a fixed order, or
DMMA tiles) and give the FP32 kernels' arithmetic ceiling."""
from __future__ import annotations

import argparse
import ctypes as C
import json
import sys

from . import build as B


def rates(iters: int = 4096) -> dict:
    lib = C.CDLL(B.build_rates())
    lib.frr_rate.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    out = {}
    for kind, name in ((0, "dfma_tflops"), (1, "dmma_tflops"), (2, "ffma_tflops")):
        t, chk = C.c_double(), C.c_double()
        if lib.frr_rate(kind, iters, C.byref(t), C.byref(chk)) != 0:
            raise RuntimeError(f"rate probe {name} failed")
        out[name] = t.value
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=4096)
    a = ap.parse_args(argv)
    print(json.dumps(rates(a.iters)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
