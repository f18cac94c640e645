"""In-tree build of the native parts: the CUDA C-ABI library (sm_103a) and
the host-side route builder used by the input generators."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB_TRANSSIM = os.path.join(HERE, "libtranssim.so")
LIB_ROUTES = os.path.join(HERE, "inputs", "libroutes.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout)
        raise RuntimeError("build failed: " + " ".join(cmd))
    return r.stdout


def build_routes_lib():
    src = os.path.join(HERE, "inputs", "routes.c")
    tmp = LIB_ROUTES + f".tmp{os.getpid()}"
    _run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", src, "-o", tmp])
    os.replace(tmp, LIB_ROUTES)


def cuda_sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def build_transsim_lib(extra_flags=()):
    """nvcc -> libtranssim.so for sm_103a, one translation unit per .cu file,
    compiled in parallel, then linked."""
    objs, procs = [], []
    os.makedirs(os.path.join(os.path.dirname(HERE), "_build"), exist_ok=True)
    for src in cuda_sources():
        obj = os.path.join(os.path.dirname(HERE), "_build", os.path.basename(src) + ".o")
        cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj, *extra_flags]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            sys.stderr.write(out)
            raise RuntimeError("build failed: " + " ".join(cmd))
    tmp = LIB_TRANSSIM + f".tmp{os.getpid()}"
    _run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIB_TRANSSIM)


def build_all():
    build_routes_lib()
    build_transsim_lib()


if __name__ == "__main__":
    build_all()
