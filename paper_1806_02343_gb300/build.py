"""Builds the in-tree CUDA library libdgmhd.so for sm_103a (and the oracle's
nothing: the oracle is pure Python). Translation units compile in parallel."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libdgmhd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# FP32 kernels of the specialised path use the hardware's approximate division,
# reciprocal square root and square root (FP64 code is unaffected)
FAST_MATH = {"dg_fast_f1.cu", "dg_fast_f2.cu", "dg_fast_f3.cu", "dg_fast_d1.cu", "dg_fast_d2.cu"}
SOURCES = ["dg_api.cu", "dg_kernels.cu", "dg_fast_f1.cu", "dg_fast_f2.cu", "dg_fast_f3.cu", "dg_fast_d1.cu", "dg_fast_d2.cu",
           "dg_cell_tc.cu", "dg_limit.cu", "dg_mlp.cu", "dg_amr.cu", "dg_noalloc.cu", "dg_probe.cu", "dg_regrid.cu", "dg_plan.cpp", "dg_basis.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
            "-I", os.path.join(HERE, "..", "include")] + ARCH


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags()
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    if src in FAST_MATH:
        cmd += ["--use_fast_math"]
    if verbose_ptxas:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "dg_mhd.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        res = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    objs = [o for o, _ in res]
    if verbose_ptxas:
        for _, log in res:
            print(log)
    tmp = LIB + ".tmp"
    cmd = [_nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
