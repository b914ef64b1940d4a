"""Build the in-tree CUDA library libpplbm.so for sm_103a with nvcc.

The translation units are compiled in parallel and linked into
``paper_2009_05264_gb300/_lib/libpplbm.so`` (static CUDA runtime, C ABI only).
``build(bounds_check=True)`` makes the test build with -DLBM_BOUNDS_CHECK in
``paper_2009_05264_gb300/_lib_bounds/libpplbm.so``: every global access of the kernels
checks its index against its buffer and a rejected access becomes LBM_EBOUNDS.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libpplbm.so")
BOUNDS_DIR = os.path.join(PKG, "_lib_bounds")
BOUNDS_LIB = os.path.join(BOUNDS_DIR, "libpplbm.so")
SOURCES = ["lbm_api.cu", "lbm_batch.cu", "lbm_f32.cu", "lbm_f64.cu", "lbm_noalloc.cu", "lbm_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(ROOT, "include", "pplbm.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(lib: str | None = None) -> bool:
    lib = lib or LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, bounds_check: bool = False) -> str:
    out_dir, lib = (BOUNDS_DIR, BOUNDS_LIB) if bounds_check else (OUT_DIR, LIB)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                    "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if ptxas_info:
        flags += ["-Xptxas", "-v"]
    if bounds_check:
        flags += ["-DLBM_BOUNDS_CHECK"]
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or ptxas_info or p.returncode != 0:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = lib + ".tmp"
    subprocess.check_call([cc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                bounds_check="--bounds-check" in sys.argv))
