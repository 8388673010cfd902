"""Build ``libvate.so`` and the measurement library ``libvate_probe.so``
in-tree with nvcc for sm_103a (B300).

    python -m paper_1812_00282_b300.build [--force] [--verbose]

The libraries are plain C ABI (include/vate*.h); the Python bindings load them
with ctypes.  Only the sm_103a cubin is generated (no PTX, no other targets).
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
SOURCES = ["vate_api.cu", "vate_kernels.cu", "vate_packed.cu", "vate_noalloc.cu", "vate_group.cu", "vate_learned.cu",
           "vate_server.cu", "vate_hostset.cu"]
PROBE_LIB = os.path.join(HERE, "libvate_probe.so")   # memory-system probes for the benchmark (include/vate_probe.h)
DEBUG_LIB = os.path.join(HERE, "libvate_debug.so")   # the checked build: the same sources with VATE_DEBUG
PROBE_SOURCES = ["vate_probe.cu"]
HEADERS = ["vate_device.cuh", "vate_device_ops.cuh", "vate_ages.cuh", "vate_launch.cuh", "vate_internal.h",
           "vate_hostset_pass.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the VATE CUDA library cannot be built")


def _stale(lib, sources) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in sources + HEADERS] + \
        [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(lib, sources, verbose, defines=()):
    tmp = lib + ".tmp%d" % os.getpid()
    extra = os.environ.get("VATE_NVCC_DEFINES", "").split() + list(defines)
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-shared", *extra,
           "-I", INCLUDE, "-I", CSRC, "-o", tmp] + [os.path.join(CSRC, f) for f in sources]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    for lib, sources, defines in ((LIB, SOURCES, ()), (PROBE_LIB, PROBE_SOURCES, ()),
                                  (DEBUG_LIB, SOURCES, ("-DVATE_DEBUG",))):
        if force or _stale(lib, sources):
            _compile(lib, sources, verbose, defines)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
