"""The kernels convert between FP32 and FP64 with integer operations (md_fpconv.cuh: a hardware
conversion runs at the FP64 pipe's rate on this part). The same header built for the host must
agree bit for bit with the host's own IEEE conversions (round to nearest, ties to even) over
random bit patterns of every class, exact ties and binade edges (tests/fpconv_check.cpp)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1812_07993_gb300", "csrc")


def test_integer_conversions_match_ieee_bit_for_bit(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "fpconv_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I" + CSRC, "-o", exe,
                    os.path.join(HERE, "fpconv_check.cpp")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
