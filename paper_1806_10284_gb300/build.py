"""Build the in-tree CUDA library ``_lib/libfame.so`` for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into one shared library with a C ABI (include/fame.h).  No cmake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libfame.so")
# the bounds-checked debug build (-DFAME_CHECK_BOUNDS), built on request
LIB_CHECK = os.path.join(OUT, "libfame_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xcompiler", "-fvisibility=hidden"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".cu", ".cpp")))


def build(verbose: bool = False, force: bool = False, check_bounds: bool = False) -> str:
    """Compile and link the library; with check_bounds the debug build with the kernels'
    bounds checks (libfame_check.so, separate objects)."""
    os.makedirs(OUT, exist_ok=True)
    lib = LIB_CHECK if check_bounds else LIB
    srcs = sources()
    deps = srcs + [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "fame.h"))
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in deps):
            return lib
    nvcc = _nvcc()
    extra = ["-DFAME_CHECK_BOUNDS"] if check_bounds else []
    suffix = ".check.o" if check_bounds else ".o"

    def compile_one(src):
        obj = os.path.join(OUT, os.path.basename(src) + suffix)
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-x", "cu", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, check_bounds="--check-bounds" in sys.argv))
