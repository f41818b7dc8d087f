"""The integer FP64 <-> FP32 conversions and the FP32-pair split used by the mixed-precision kernels
(paper_1208_6387_gb300/csrc/ds.cuh), compiled for the host with g++ and checked against the C++ conversions:
FP32 -> FP64 exact, FP64 -> FP32 rounded to nearest, pairs within 2^-48 (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1208_6387_gb300", "csrc")


def test_integer_conversions_match_the_cpp_conversions(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "ds_conversions")
    subprocess.run([cxx, "-O2", "-std=c++17", "-frounding-math", "-I", CSRC,
                    os.path.join(HERE, "host", "ds_conversions.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
