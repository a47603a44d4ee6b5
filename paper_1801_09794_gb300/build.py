"""Builds the CUDA library libfeast_nl.so in-tree for sm_103a (nvcc, no cmake).

Translation units are compiled in parallel; the link is skipped when the
library is newer than every source and header.
"""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = ["k_dense.cu", "k_lu.cu", "k_reduced.cu", "k_ozaki.cu", "k_cgemm_tc.cu", "feast_nl.cu",
           "noalloc.cu", "server.cpp"]
HEADERS = [os.path.join(CSRC, "internal.h"), os.path.join(CSRC, "tc_common.cuh"), os.path.join(CSRC, "cgemm_tile.cuh"), os.path.join(ROOT, "include", "feast_nl.h")]
LIB = os.path.join(HERE, "libfeast_nl.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        p = os.path.join(cand, "bin", "nvcc") if cand else ""
        if p and os.path.exists(p):
            return p
    p = shutil.which("nvcc")
    if not p:
        raise RuntimeError("nvcc not found (set CUDA_HOME)")
    return p


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra_flags=()):
    """Compile every CUDA translation unit and link libfeast_nl.so; returns its path."""
    nvcc = _nvcc()
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    objs = [os.path.join(objdir, os.path.splitext(s)[0] + ".o") for s in SOURCES]

    def compile_one(pair):
        src, obj = pair
        if not force and not _stale(obj, [src] + HEADERS):
            return None
        cmd = [nvcc, "-c", src, "-o", obj] + ARCH + FLAGS + list(extra_flags)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        return r.stderr if verbose else None

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        for msg in ex.map(compile_one, zip(srcs, objs)):
            if msg:
                print(msg)
    if force or _stale(LIB, objs):
        cmd = [nvcc, "-shared", "-o", LIB] + objs + ARCH + ["-Xcompiler", "-fPIC", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
