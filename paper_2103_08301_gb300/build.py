"""Build the solver's shared library (liblbm.so) in-tree for sm_103a.

Seven translation units, compiled in parallel and linked with nvcc:
  csrc/lbm_api.cu     - single-channel C ABI and the step kernels (nvcc, -gencode sm_103a)
  csrc/lbm_big.cu     - the step kernels with 64-bit population offsets (grids of 9 pitch ny >= 2^31)
  csrc/lbm_batch.cu   - batched multi-channel sweep (nvcc)
  csrc/lbm_adjoint.cu - discrete adjoint with checkpoint-and-recompute (nvcc)
  csrc/lbm_mask.cu    - general wall geometry (per-node solid mask) step kernels (nvcc)
  csrc/lbm_inplace.cu - in-place (AA pattern) single-context step kernels (nvcc)
  csrc/lbm_host.cpp   - host FP64 thermodynamics, initial profiles, plug analysis (g++)
Run as ``python -m paper_2103_08301_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = ["lbm_api.cu", "lbm_big.cu", "lbm_batch.cu", "lbm_adjoint.cu", "lbm_mask.cu", "lbm_inplace.cu", "lbm_host.cpp",
           "lbm_kernels.cuh", "lbm_rows2.cuh", "lbm_tile.cuh", "lbm_internal.h"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(INCLUDE, "lbm.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, out: str | None = None) -> str:
    """Compile liblbm.so (or `out`) if missing or out of date; return its path."""
    lib = out or LIB
    if not force and out is None and not _stale():
        return LIB
    bdir = BUILD if out is None else out + ".build"
    os.makedirs(bdir, exist_ok=True)
    api_o = os.path.join(bdir, "lbm_api.o")
    batch_o = os.path.join(bdir, "lbm_batch.o")
    adj_o = os.path.join(bdir, "lbm_adjoint.o")
    host_o = os.path.join(bdir, "lbm_host.o")
    mask_o = os.path.join(bdir, "lbm_mask.o")
    big_o = os.path.join(bdir, "lbm_big.o")
    aa_o = os.path.join(bdir, "lbm_inplace.o")
    extra = os.environ.get("LBM_NVCC_FLAGS", "").split()  # tuning experiments, e.g. -DLBM_STAGE_AHEAD=2

    def nvcc(src, obj):
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
               "-I", CSRC, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        return cmd

    gxx = ["g++", "-O2", "-std=c++17", "-fPIC", "-I", INCLUDE, "-I", CSRC, "-c",
           os.path.join(CSRC, "lbm_host.cpp"), "-o", host_o]
    with ThreadPoolExecutor(7) as ex:
        outs = list(ex.map(_run, [nvcc("lbm_api.cu", api_o), nvcc("lbm_big.cu", big_o), nvcc("lbm_batch.cu", batch_o),
                                  nvcc("lbm_adjoint.cu", adj_o), nvcc("lbm_mask.cu", mask_o),
                                  nvcc("lbm_inplace.cu", aa_o), gxx]))
    if verbose:
        for o in outs[:6]:
            print(o)
    tmp = lib + f".tmp{os.getpid()}"
    _run([NVCC, *ARCH, "-shared", "-o", tmp, api_o, big_o, batch_o, adj_o, mask_o, aa_o, host_o, "-lcudart"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
