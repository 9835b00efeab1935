"""Builds the in-tree shared library ``libhradon.so`` for sm_103a.

Every ``csrc/*.cu`` (kernels, the no-alloc entry point, the sparse-inversion
solver) with nvcc (``-gencode arch=compute_103a,code=sm_103a``) and
``csrc/plan.cpp`` with the host compiler (``-ffp-contract=off`` keeps the FP64
geometry identical on x86-64 and aarch64 hosts), compiled in parallel. No
torch, no cmake.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libhradon.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _sources():
    return [os.path.join(CSRC, n) for n in sorted(os.listdir(CSRC))
            if n.endswith((".cu", ".cpp", ".h", ".cuh"))] + [os.path.join(INCLUDE, "hradon.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    inc = ["-I", CSRC, "-I", INCLUDE, "-I", os.path.join(cuda, "include")]
    cmds, objs = [], []
    for name in sorted(n for n in os.listdir(CSRC) if n.endswith(".cu")):
        obj = os.path.join(bdir, name[:-3] + ".o")
        cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xcompiler", "-ffp-contract=off", *inc, "-c", os.path.join(CSRC, name), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        cmds.append(cmd)
        objs.append(obj)
    po = os.path.join(bdir, "plan.o")
    cmds.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall", *inc, "-c",
                 os.path.join(CSRC, "plan.cpp"), "-o", po])
    objs.append(po)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose or ptxas_info:
            sys.stderr.write(r.stdout + r.stderr)

    with ThreadPoolExecutor(len(cmds)) as ex:
        list(ex.map(run, cmds))
    tmp = LIB + f".tmp{os.getpid()}"
    run([nvcc, *ARCH, "-shared", *objs, "-o", tmp, "-L", os.path.join(cuda, "lib64"), "-lcudart", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
