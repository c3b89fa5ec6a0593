"""Build libsdd.so in-tree: CUDA sources for sm_103a with nvcc, host C++ with g++.

Translation units compile in parallel; the result lands next to this file.  Set
SDD_PTXAS_VERBOSE=1 to see register / shared-memory usage per kernel.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsdd.so")
ROOT = os.path.dirname(HERE)

CUDA_SOURCES = ["api.cu", "render_kernels.cu", "photon.cu", "bundle_kernels.cu", "graph_kernels.cu", "noalloc.cu", "persistent.cu", "persistent_bundle.cu", "tile.cu", "mlp.cu", "surrogate_render.cu"]
CXX_SOURCES = ["scene_build.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The persistent kernel reads, within one launch, ray / hit / queue / path data that other
# blocks (other SMs) wrote before a grid barrier; plain global loads are made to bypass the
# SM's L1 (cache at L2 only) so that no stale L1 line is read.  Read-only scene data is
# fetched with __ldg and keeps its caching.
PER_FILE_FLAGS = {"persistent.cu": ["-Xptxas", "-dlcm=cg"], "persistent_bundle.cu": ["-Xptxas", "-dlcm=cg"]}


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.exists(os.path.join(home, "bin", "nvcc")):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "sdd.h"))
    jobs = []
    objs = []
    ptxas_v = ["-Xptxas", "-v"] if os.environ.get("SDD_PTXAS_VERBOSE") else []
    for f in CUDA_SOURCES:
        src = os.path.join(SRC, f)
        obj = os.path.join(OUT_DIR, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", SRC, "-I", os.path.join(ROOT, "include"), *ptxas_v, *PER_FILE_FLAGS.get(f, []),
                   "-c", src, "-o", obj]
            jobs.append(cmd)
    for f in CXX_SOURCES:
        src = os.path.join(SRC, f)
        obj = os.path.join(OUT_DIR, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-I", SRC, "-I", os.path.join(cuda, "include"),
                   "-c", src, "-o", obj]
            jobs.append(cmd)
    procs = [(cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
             for cmd in jobs]
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0 or ptxas_v:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("libsdd build failed:\n" + "\n".join(failed))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp"
        subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
