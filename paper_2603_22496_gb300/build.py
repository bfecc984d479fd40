"""Build the in-tree shared library ``_build/libkkbeam.so`` (sm_103a only).

Each translation unit is compiled by nvcc in parallel, then linked with
``nvcc -shared``.  Run as ``python -m paper_2603_22496_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libkkbeam.so")
# bounds-checked variant (-DKK_DEBUG_BOUNDS): every gather index is checked and
# failures are counted on the device (kk_debug_bounds); built on demand
LIB_BOUNDS = os.path.join(BUILD, "libkkbeam_bounds.so")
VARIANTS = {"": (BUILD, LIB, []), "bounds": (os.path.join(BUILD, "bounds"), LIB_BOUNDS, ["-DKK_DEBUG_BOUNDS"])}
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found (CUDA toolkit required to build the library)")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith(".cu") or f.endswith(".cpp"))


def _deps_mtime():
    files = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, extra, outdir: str = BUILD) -> str:
    obj = os.path.join(outdir, os.path.basename(src) + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= _deps_mtime():
        return obj
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + list(extra) + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None,
          variant: str = "") -> str:
    """Compile the library ('' = the product library; 'bounds' = the
    bounds-checked variant) and return its path."""
    outdir, lib, vflags = VARIANTS[variant]
    os.makedirs(outdir, exist_ok=True)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    if force:
        for f in os.listdir(outdir):
            if f.endswith(".o"):
                os.remove(os.path.join(outdir, f))
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + vflags
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, outdir), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv,
                variant="bounds" if "--bounds" in sys.argv else ""))
