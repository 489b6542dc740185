"""Build libcola.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each CUDA translation unit is compiled in its own nvcc process (in parallel)
and the objects are linked into paper_2302_00850_gb300/_build/libcola.so with
the CUDA runtime linked statically, so the library depends only on the
driver.  Usage: python -m paper_2302_00850_gb300.build [--force] [--bounds]
(--bounds: the debug build with index checks, in _build_bounds/).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libcola.so")
SOURCES = ["dslash.cu", "dslash_clover.cu", "clover.cu", "clover_force.cu", "blas.cu", "pack.cu", "force.cu", "gauge.cu", "hmc.cu",
           "solver.cu", "multishift.cu", "eig.cu", "api.cu", "noalloc.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcola")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "cola.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps())


def _compile(src: str, extra, out_dir: str) -> str:
    obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


BOUNDS_DIR = os.path.join(PKG, "_build_bounds")


def build_bounds(force: bool = False) -> str:
    """The debug build with every computed index checked (-DCOLA_BOUNDS), in _build_bounds/;
    load it with COLA_LIB=<returned path>."""
    return build(force=force, extra=["-DCOLA_BOUNDS"], out_dir=BOUNDS_DIR)


def build(force: bool = False, verbose: bool = False, extra=(), out_dir: str | None = None) -> str:
    """Compile every translation unit and link libcola.so; returns its path.

    out_dir (default the package's _build folder) and extra nvcc flags allow
    side-by-side builds of tuning variants.
    """
    out_dir = out_dir or BUILD
    lib = os.path.join(out_dir, "libcola.so")
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    flags = list(extra) + (["-Xptxas", "-v"] if verbose else [])
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, flags, out_dir), SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    if "--bounds" in sys.argv:
        path = build_bounds(force="--force" in sys.argv)
    else:
        path = build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(path)
