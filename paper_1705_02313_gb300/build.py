"""Builds libpg.so (the CUDA solver behind include/pg.h) for sm_103a, and
libpggen.so (the multithreaded host generator of random games).

Each translation unit under csrc/ is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and the objects
are linked into ``paper_1705_02313_gb300/libpg.so`` (CUDA runtime linked
statically); ``csrc/gen_host.c`` is compiled by the host C compiler. Each
library is rebuilt only when one of its sources is newer than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpg.so")
GEN_LIB = os.path.join(HERE, "libpggen.so")
GEN_SRC = os.path.join(CSRC, "gen_host.c")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def nvcc():
    for cand in [os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"]:
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "pg.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build_gen(force: bool = False) -> str:
    """Compiles the host generator (plain C, no CUDA)."""
    if not force and os.path.exists(GEN_LIB) and os.path.getmtime(GEN_LIB) >= max(
            os.path.getmtime(GEN_SRC), os.path.getmtime(__file__)):
        return GEN_LIB
    cc = os.environ.get("CC", "gcc")
    tmp = GEN_LIB + ".%d.tmp" % os.getpid()
    cmd = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", GEN_SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("host generator build failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, GEN_LIB)
    return GEN_LIB


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    build_gen(force)
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(OUT, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(extra), extra=extra))
