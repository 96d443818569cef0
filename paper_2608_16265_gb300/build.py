"""Builds libexa.so (the C-ABI library) in-tree for sm_103a.

Four translation units compiled in parallel: exa_api.cu, exa_sort.cu and exa_probe.cu with nvcc
(-gencode arch=compute_103a,code=sm_103a), exa_lower.cpp with g++; linked against the shared CUDA
runtime and NVRTC (no libcuda link dependency, so the library also loads on hosts without a GPU
driver).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "libexa.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libexa.so")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp", ".h", ".inc")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = _sources() + [os.path.join(INCLUDE, h) for h in os.listdir(INCLUDE)] + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    os.makedirs(OBJDIR, exist_ok=True)
    jobs = []
    common = ["-O3", "-std=c++17", "-I", INCLUDE]
    for f in ("exa_api.cu", "exa_sort.cu", "exa_probe.cu"):
        out = os.path.join(OBJDIR, f + ".o")
        jobs.append((out, [nvcc, *ARCH, *common, "-lineinfo", "-Xcompiler", "-fPIC", "-c",
                           os.path.join(CSRC, f), "-o", out]))
    out = os.path.join(OBJDIR, "exa_lower.cpp.o")
    jobs.append((out, ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE,
                       "-I", os.path.join(cuda, "include"), "-c", os.path.join(CSRC, "exa_lower.cpp"),
                       "-o", out]))
    procs = []
    for out, cmd in jobs:
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for cmd, p in procs:
        log, _ = p.communicate()
        if p.returncode != 0:
            errors.append(" ".join(cmd) + "\n" + log.decode(errors="replace"))
        elif verbose and log:
            print(log.decode(errors="replace"), file=sys.stderr)
    if errors:
        raise RuntimeError("libexa build failed:\n" + "\n".join(errors))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *[o for o, _ in jobs],
            "-L", os.path.join(cuda, "lib64"), "-lnvrtc"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("libexa link failed:\n" + " ".join(link) + "\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
