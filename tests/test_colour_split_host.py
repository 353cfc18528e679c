"""The colour-split index maps of the FP32 storage (dense and oct levels),
compiled as host C++ from the header the kernels include: bijections, the
red-black planes, the inverse map and the six periodic neighbours."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_colour_split_index_maps():
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "colour_split_check")
        subprocess.run(["g++", "-std=c++17", "-O1", os.path.join(HERE, "colour_split_check.cpp"),
                        "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == 0
