"""Build ``libvate.so`` in-tree with nvcc for sm_103a (B300).

    python -m paper_1812_00282_b300.build [--force] [--verbose]

The library is plain C ABI (include/vate.h); the Python binding loads it with
ctypes.  Only the sm_103a cubin is generated (no PTX, no other targets).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libvate.so")
SOURCES = ["vate_api.cu", "vate_kernels.cu", "vate_packed.cu", "vate_probe.cu", "vate_noalloc.cu", "vate_group.cu", "vate_learned.cu", "vate_server.cu"]
HEADERS = ["vate_device.cuh", "vate_device_ops.cuh", "vate_ages.cuh", "vate_launch.cuh", "vate_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the VATE CUDA library cannot be built")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + \
        [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    extra = os.environ.get("VATE_NVCC_DEFINES", "").split()
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-shared", *extra,
           "-I", INCLUDE, "-I", CSRC, "-o", tmp] + [os.path.join(CSRC, f) for f in SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
