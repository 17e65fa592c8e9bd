"""The library's own sin/cos(pi x) (phasor seeds of the NDFT kernels) against
CUDA's sincospif on 2^24 arguments in [-1, 1]: within 3 units of the last
place of sincospif's value (itself within 1 ulp of exact), i.e. within the
2 ulp design bound of the polynomial plus sincospif's own error."""
import os
import re
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_sincospi_reduced_matches_sincospif(tmp_path):
    exe = str(tmp_path / "sincospi_check")
    src = os.path.join(HERE, "sincospi_check.cu")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I" + os.path.join(ROOT, "include"),
                    "-I" + os.path.join(ROOT, "paper_2603_08386_gb300", "csrc"), src, "-o", exe],
                   check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    m = re.search(r"max_sin_ulp ([0-9.]+) max_cos_ulp ([0-9.]+) err (.*)", out)
    assert m, out
    assert m.group(3).strip() == "no error"
    assert float(m.group(1)) <= 3.0 and float(m.group(2)) <= 3.0, out
