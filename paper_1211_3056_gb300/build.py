"""Build the CUDA libraries in-tree for sm_103a.

libtmd.so: three translation units (host planning/tables, kernels, C-ABI
glue), the search library of include/tmd.h.  libtmd_probe.so: the pipe-rate
probe of include/tmd_probe.h (measurement support, not the search path).
The four units are compiled in parallel with nvcc; both shared objects land
next to this file.  `python -m paper_1211_3056_gb300.build` runs it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libtmd.so")
PROBE_LIB = os.path.join(HERE, "libtmd_probe.so")
OBJ = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"]
LIB_SOURCES = ["host.cpp", "kernels.cu", "api.cu"]
PROBE_SOURCES = ["probe.cu"]
SOURCES = LIB_SOURCES + PROBE_SOURCES


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtmd.so")
    return cand


def _newer(src_paths, out) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(p) > t for p in src_paths)


def build(force: bool = False, verbose: bool = False) -> str:
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(os.path.dirname(HERE), "include", h) for h in ("tmd.h", "tmd_probe.h")]
    if not force and not _newer(deps, LIB) and not _newer(deps, PROBE_LIB):
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(OBJ, src + ".o")
        cmd = [cc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = dict(zip(SOURCES, ex.map(compile_one, SOURCES)))

    def link(out, srcs, extra):
        tmp = out + ".tmp"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *[objs[x] for x in srcs], *extra]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"linking {os.path.basename(out)} failed:\n" + r.stderr)
        os.replace(tmp, out)

    link(LIB, LIB_SOURCES, ["-lpthread"])
    link(PROBE_LIB, PROBE_SOURCES, [])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
