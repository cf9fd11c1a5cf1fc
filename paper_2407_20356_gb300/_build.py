"""Build the CUDA library libxpcs.so (sm_103a) in-tree.

Every translation unit is compiled in parallel with nvcc for sm_103a only, then linked
into ``paper_2407_20356_gb300/lib/libxpcs.so``.  No torch types cross the library's ABI.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libxpcs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def build_library(verbose: bool = False, extra=()) -> str:
    nvcc = _nvcc()
    obj = os.path.join(LIBDIR, "obj")
    os.makedirs(obj, exist_ok=True)
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include"),
                    "--expt-relaxed-constexpr", *extra]
    srcs = sources()
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(ROOT, "include", "xpcs.h"))
    newest_hdr = max(os.path.getmtime(h) for h in hdrs)

    def one(src):
        o = os.path.join(obj, os.path.basename(src)[:-3] + ".o")
        if os.path.exists(o) and os.path.getmtime(o) > max(os.path.getmtime(src), newest_hdr) and not extra:
            return o
        cmd = [nvcc, *flags, "-c", src, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return o

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(one, srcs))
    cmd = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-lcusolver", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build_library(verbose=True))
