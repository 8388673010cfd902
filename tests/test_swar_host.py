"""The SWAR forms of CheckAT (Algorithm 1), the census distance (Eq. 5) and
fast PreserveAT (Algorithm 3) used by the kernels, checked on the CPU against
their scalar forms for every k <= 63, ACT and k' (tests/swar_host_check.cu,
compiled for the host from the library's device header)."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_swar_arithmetic_matches_scalar_forms(tmp_path):
    from paper_1812_00282_b300.build import nvcc
    exe = str(tmp_path / "swar_check")
    subprocess.check_call([nvcc(), "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1812_00282_b300", "csrc"),
                           "-o", exe, os.path.join(HERE, "swar_host_check.cu")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("OK")
