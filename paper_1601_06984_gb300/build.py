"""Build liblbm.so in-tree: CUDA kernels for sm_103a (nvcc) and the host mesh
builder / C ABI (g++ with OpenMP), compiled in parallel and linked with nvcc."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "liblbm.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

CU = ["kernels_fp64.cu", "kernels_fp32dev.cu", "kernels_bf16dev.cu", "reduce_noalloc.cu",
      "adjoint_fp64.cu", "adjoint_fp32dev.cu", "adjoint_bf16dev.cu", "probe.cu"]
CPP = ["mesh.cpp", "api.cpp", "adjoint.cpp", "partition.cpp"]


def _cuda_home() -> str:
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _sources():
    return [os.path.join(CSRC, f) for f in CU + CPP + ["kernels.cuh", "adjoint.cuh", "lbm_internal.h",
                                                      "lbm_ctx.h"]] + [
        os.path.join(INCLUDE, "lbm.h")]


def up_to_date() -> bool:
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + INCLUDE, "-I" + CSRC]
    cmds = []
    for f in CU:
        obj = os.path.join(BUILD, f + ".o")
        cmds.append([nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
                     "-c", os.path.join(CSRC, f), "-o", obj])
    for f in CPP:
        obj = os.path.join(BUILD, f + ".o")
        cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-fopenmp", "-Wall", *inc,
                     "-I" + os.path.join(cuda, "include"), "-c", os.path.join(CSRC, f), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        list(ex.map(run, cmds))
    objs = [os.path.join(BUILD, f + ".o") for f in CU + CPP]
    tmp = OUT + ".tmp"
    run([nvcc, ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp", "-cudart", "shared"])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
