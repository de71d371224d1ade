"""Build the LBRS CUDA library (liblbrs.so) in-tree for sm_103a.

Six translation units compiled in parallel with nvcc, then linked into one
shared library with the CUDA runtime linked statically:

  csrc/lbrs_kernels_f64.cu  FP64 kernels, -fmad=false (rounding as written)
  csrc/lbrs_kernels_f32.cu  FP32 step kernels
  csrc/lbrs_kernels_f16.cu  D2Q4 step with FP16 non-equilibrium storage
  csrc/lbrs_runtime.cu      host C ABI (include/lbrs.h)
  csrc/lbrs_noalloc.cu      diagnostics variant with static scratch, -fmad=false
  csrc/lbrs_batch_runtime.cu host runtime of the batched tubes

The bounds-checked variant (-DLBRS_DEBUG: every checked kernel index that leaves
its buffer is recorded and replaced by 0, see lbrs_debug_check in include/lbrs.h)
builds into _build_debug/ as liblbrs_debug.so; load it with LBRS_LIBRARY.

Usage: python -m paper_1504_07034_gb300.build [--force] [--debug]
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"
LIB = PKG / "liblbrs.so"
BUILD_DEBUG = PKG / "_build_debug"
LIB_DEBUG = PKG / "liblbrs_debug.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "-Xptxas", "-v", "-I", str(INCLUDE), "-I", str(CSRC)]
UNITS = {
    "lbrs_kernels_f64.cu": ["-fmad=false"],
    "lbrs_kernels_f32.cu": [],
    "lbrs_kernels_f16.cu": [],
    "lbrs_runtime.cu": [],
    "lbrs_noalloc.cu": ["-fmad=false"],
    "lbrs_batch_runtime.cu": [],
}
HEADERS = [CSRC / "lbrs_kernels.cuh", CSRC / "lbrs_batch.cuh", CSRC / "lbrs_launch.h", INCLUDE / "lbrs.h"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbrs.so")
    return exe


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(d).stat().st_mtime > t for d in deps)


def _compile(unit: str, extra, bdir: Path = BUILD) -> Path:
    src = CSRC / unit
    obj = bdir / (unit + ".o")
    log = bdir / (unit + ".ptxas.log")
    cmd = [nvcc(), *ARCH, *COMMON, *extra, "-c", str(src), "-o", str(obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    log.write_text(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr[-4000:]}")
    return obj


def build(force: bool = False, debug: bool = False) -> Path:
    bdir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    flags = ["-DLBRS_DEBUG"] if debug else []
    bdir.mkdir(parents=True, exist_ok=True)
    todo = [(u, x) for u, x in UNITS.items()
            if force or _stale(bdir / (u + ".o"), [CSRC / u, *HEADERS])]
    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        list(ex.map(lambda ux: _compile(ux[0], [*ux[1], *flags], bdir), todo))
    objs = [bdir / (u + ".o") for u in UNITS]
    if force or todo or _stale(lib, objs):
        tmp = lib.with_name(f"{lib.stem}.{os.getpid()}.tmp.so")
        cmd = [nvcc(), *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, debug="--debug" in sys.argv))
