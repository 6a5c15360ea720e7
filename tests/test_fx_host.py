"""The fixed-point / double-float helpers of the FP64-free particle kernel,
compiled for the host and checked against long double on 2M random inputs:
FP64 -> fixed point rounds to nearest, fixed point -> FP64 is IEEE
round-to-nearest-even, the double-float splits, products, sums and square
roots keep 44+ bits, and the FP64-free conversions between FP64, FP32 and
the stored double-float pairs are bit-identical to the FP64 expressions."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fx_helpers_on_host(tmp_path):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "fxcheck"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-x", "c++",
                           os.path.join(HERE, "fx_host_check.cpp"), "-o", str(exe), "-lm"])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "bad 0" in out.stdout
