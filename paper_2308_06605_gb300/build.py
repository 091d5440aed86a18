"""Build the C-ABI CUDA library `lib/libfr.so` in-tree with nvcc for sm_103a.

Translation units are compiled in parallel, then linked against the shared CUDA runtime (the
same libcudart PyTorch loads).  Usage: `python -m paper_2308_06605_gb300.build`.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libfr.so")
SOURCES = ["fr_mesh.cpp", "fr_tri.cpp", "fr_curved.cpp", "fr_part.cpp", "fr_kernels.cu", "fr_tc.cu", "fr_vcjh.cu", "fr_prism.cu", "fr_api.cu", "fr_probe.cu",
           "fr_static.cu", "fr_batch.cu", "fr_mlp.cu", "fr_project.cu"]
# The batched stage kernel is compiled once per (precision, block size) so the variants build in parallel.
VARIANTS = [("fr_batch_kernel.cu", f"m{m}_b{b}", [f"-DFRX_BATCH_MIXED={m}", f"-DFRX_BATCH_BLOCK={b}"])
            for m in (0, 1) for b in (256, 512)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def cuda_libdir() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    common = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC, *extra]

    # An object is rebuilt when it is older than its source or than any header (headers are shared).
    headers = [os.path.join(d, f) for d in (CSRC, os.path.join(ROOT, "include")) for f in os.listdir(d)
               if f.endswith((".h", ".hpp", ".cuh"))]
    newest_header = max(os.path.getmtime(h) for h in headers)

    def compile_one(unit):
        src, tag, flags = unit if isinstance(unit, tuple) else (unit, "", [])
        obj = os.path.join(objdir, src + (("." + tag) if tag else "") + ".o")
        if (not verbose and not extra and os.path.exists(obj) and os.path.exists(LIB)
                and os.path.getmtime(obj) > max(newest_header, os.path.getmtime(os.path.join(CSRC, src)))):
            return obj
        cmd = common + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    units = VARIANTS + SOURCES          # slowest first
    with ThreadPoolExecutor(max_workers=len(units)) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath," + cuda_libdir()]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
