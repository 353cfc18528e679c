"""The double-float primitives of the mixed form, compiled as host C++ and
checked against long double on seeded operands: conversion from FP64, add,
multiply, e^x on [-40, 40] and 1/sqrt(x) on [e^-30, e^30]; the conversions
that work on the bit patterns (FP64 <-> FP32 and double-float) against the
C casts, bit for bit, including values next to rounding ties.  The FP64-accurate
residual needs about 1e-12 relative; double-float carries ~48 bits."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_dfloat_primitives_accuracy():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "dfloat_check")
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off",
                        os.path.join(HERE, "dfloat_check.cpp"), "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    conv, add, mul, ex, rsq = (float(v) for v in out[:5])
    assert int(out[5]) == 0   # integer-pipe conversions match the casts bit for bit
    assert conv <= 2e-15      # FP64 -> pair -> FP64 keeps ~49 bits
    assert add <= 5e-14
    assert mul <= 5e-14
    assert ex <= 1e-13
    assert rsq <= 1e-13
