"""Compile the CUDA library (sm_103a) into paper_1503_06726_gb300/_build/liblbib.so.

Each .cu translation unit is compiled in parallel with nvcc for
compute_103a/sm_103a only, then linked into one shared library that exports
the C ABI of include/lbib.h.  Run ``python -m paper_1503_06726_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbib.so")
# the checking build (-DLBIB_CHECK): every vector, atomic and indexed access of
# the hot kernels tests its address first, records a failure in the context's
# diagnostic words and skips the access; selected by LBIB_CHECK=1
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(BUILD_CHECK, "liblbib_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), check: bool = False) -> str:
    """Compile the library (check=True: the checking build, -DLBIB_CHECK)."""
    build_dir = BUILD_CHECK if check else BUILD
    lib = LIB_CHECK if check else LIB
    if check:
        extra = tuple(extra) + ("-DLBIB_CHECK",)
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(ROOT, "include", "lbib.h"))
    srcs = sources()
    objs = [os.path.join(build_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    nv = nvcc()

    def comp(src, obj):
        if not force and not _stale(obj, [src] + headers):
            return None
        cmd = [nv, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return r.stderr if verbose else None

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        logs = list(ex.map(lambda so: comp(*so), zip(srcs, objs)))
    if verbose:
        for l in logs:
            if l:
                print(l, file=sys.stderr)
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nv, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                check="--check" in sys.argv))
