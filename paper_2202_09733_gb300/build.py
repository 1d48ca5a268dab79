"""Build the frpmg CUDA library (libfrpmg.so) in-tree for sm_103a.

Translation units:
  csrc/kernels64.cu   FP64 kernels, nvcc -fmad=false (only explicit fma contractions)
  csrc/kernels32.cu   FP32 kernels of the mixed-precision preconditioner
  csrc/kernelsad.cu   FP32 forward-mode (dual-number) residual for the FP32 element blocks
  csrc/lib.cu         C ABI and host orchestration
  csrc/noalloc.cu     fr_residual_noalloc (stage scratch in a fixed device array)
  csrc/mlp.cu         per-element BF16 MLP for the Newton initial guess
  csrc/batch_kernels.cu  segmented (per-problem) vector kernels of the batched solver
  csrc/mbnk.cu        matrix-based Newton-Krylov smoother of the coarsest pMG level
  csrc/lu_tc.cu       batched LU of the FP32 element blocks, trailing updates on tcgen05
  csrc/padapt.cu      p-adaptation: spectral-decay indicator and marking (Sec. 3.3)
  csrc/host_tables.c  binary128 operator tables         (gcc -ffp-contract=off)
  csrc/host_geometry.c geometric factors, connectivity  (gcc -ffp-contract=off)
build_rates() compiles csrc/rates.cu (pipe-rate microbenchmarks) into librates.so.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfrpmg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the frpmg CUDA library cannot be built")


def _units():
    nv = _nvcc()
    inc = ["-I", os.path.join(HERE, "..", "include"), "-I", CSRC]
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"] + inc
    return [
        ([nv] + common + ["-fmad=false", "-c"], "kernels64.cu"),
        ([nv] + common + ["-c"], "kernels32.cu"),
        ([nv] + common + ["-c"], "kernelsad.cu"),
        ([nv] + common + ["-c"], "lib.cu"),
        ([nv] + common + ["-c"], "noalloc.cu"),
        ([nv] + common + ["-c"], "mlp.cu"),
        ([nv] + common + ["-fmad=false", "-c"], "batch_kernels.cu"),
        ([nv] + common + ["-fmad=false", "-c"], "mbnk.cu"),
        ([nv] + common + ["-c"], "lu_tc.cu"),
        ([nv] + common + ["-fmad=false", "-c"], "padapt.cu"),
        (["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC"] + inc + ["-c"], "host_tables.c"),
        (["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC"] + inc + ["-c"], "host_geometry.c"),
    ]


def _sources():
    out = []
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".c", ".h")):
            out.append(os.path.join(CSRC, f))
    out.append(os.path.join(HERE, "..", "include", "frpmg.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    units = _units()
    objs = []

    def run(u):
        cmd, src = u
        obj = os.path.join(BUILD, src + ".o")
        full = cmd + [os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(full, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compiling {src} failed:\n{' '.join(full)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(units)) as ex:
        objs = list(ex.map(run, units))
    tmp = LIB + f".{os.getpid()}.tmp"
    link = [_nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + \
        ["-Xlinker", "-rpath=/usr/local/cuda/lib64"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking failed:\n{' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


RATES_LIB = os.path.join(HERE, "librates.so")


def build_rates(force: bool = False) -> str:
    """The pipe-rate microbenchmarks (csrc/rates.cu) as their own library."""
    src = os.path.join(CSRC, "rates.cu")
    if not force and os.path.exists(RATES_LIB) and os.path.getmtime(RATES_LIB) >= os.path.getmtime(src):
        return RATES_LIB
    tmp = RATES_LIB + f".{os.getpid()}.tmp"
    cmd = [_nvcc()] + ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
                              "-o", tmp, src]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling rates.cu failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, RATES_LIB)
    return RATES_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
