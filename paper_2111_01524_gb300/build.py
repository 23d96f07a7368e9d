"""Build of the CUDA library ``_lib/libgvof.so`` (sm_103a, in-tree).

Each translation unit is compiled in parallel with nvcc, then linked into
one shared library with a plain C ABI (``include/vof.h``).
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libgvof.so")
UNITS = ["capi.cu", "k_setup.cu", "k_sweep.cu", "k_recon.cu", "k_flux.cu", "k_init.cu", "noalloc.cu", "halo.cu",
         "server.cu", "mesh_host.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    deps.append(os.path.join(HERE, "..", "include", "vof.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp",
              "-I", os.path.join(HERE, "..", "include")]
    if os.environ.get("GVOF_PTXAS_V"):
        common += ["-Xptxas", "-v"]

    def compile_one(u):
        src = os.path.join(SRC, u)
        obj = os.path.join(OUT, u + ".o")
        if u.endswith(".cpp"):
            cmd = [nvcc, "-x", "c++", "-c", src, "-o", obj] + common
        else:
            cmd = [nvcc, "-c", src, "-o", obj] + ARCH + common
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {u}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, "-shared", "-o", tmp] + ARCH + objs + ["-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
