"""Build libchfsi.so in-tree for sm_103a (GB300).

Compiles the translation units of ``csrc/`` in parallel with nvcc / g++ and
links them with cuSOLVER into ``paper_1903_10959_gb300/libchfsi.so``.  Only
one ``-gencode`` (compute_103a -> sm_103a) is emitted.  Object files go to
``_build/`` beside the package.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libchfsi.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_SOURCES = ["kernels_fp64.cu", "kernels_tc.cu", "kernels_mf.cu", "api.cu", "batch.cu", "server.cu",
                "density.cu", "scf.cu", "kpoint.cu"]
CXX_SOURCES = ["mesh.cpp", "partition.cpp"]


def _sources():
    return [os.path.join(CSRC, f) for f in CUDA_SOURCES + CXX_SOURCES]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = _sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    deps.append(os.path.join(ROOT, "include", "chfsi.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libchfsi.so; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    jobs, objs = [], []
    for f in CUDA_SOURCES:
        obj = os.path.join(BUILD, f.replace(".cu", ".o"))
        cmd = [NVCC, *GENCODE, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp",
               *inc, "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append(cmd)
        objs.append(obj)
    for f in CXX_SOURCES:
        obj = os.path.join(BUILD, f.replace(".cpp", ".o"))
        cxx = shutil.which("g++") or "c++"
        cmd = [cxx, "-O3", "-std=c++17", "-fPIC", "-fopenmp", *inc,
               "-I" + os.path.join(CUDA_HOME, "include"), "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append(cmd)
        objs.append(obj)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c in jobs]
    errors = []
    for c, p in zip(jobs, procs):
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(" ".join(c) + "\n" + out.decode(errors="replace"))
        elif verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("libchfsi build failed:\n" + "\n".join(errors))
    tmp = LIB + ".tmp"
    link = [NVCC, *GENCODE, "-shared", "-o", tmp, *objs, "-lcusolver", "-lcublas", "-lcudart",
            "-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libchfsi link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
