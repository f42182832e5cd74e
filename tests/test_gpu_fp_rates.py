"""Issue rates of the arithmetic the float kernels are designed around, on
the GPU the tests run on (tests/probes/fp_rates.cu, built with nvcc here).
The float64 elimination of the column solve is the one float64 part of the
mixed-precision step because float64 FMA issues far below float32 FMA on
this part, and its float32 <-> float64 conversions run on the integer ALU
because the conversion instruction issues at the float64 FMA rate."""

import os
import shutil
import subprocess
import tempfile

import pytest

from conftest import report_dir

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_float64_issue_rates():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "fp_rates")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, "probes", "fp_rates.cu")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rates = {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}
    if report_dir():
        with open(os.path.join(report_dir(), "fp_rates.txt"), "w") as f:
            f.write(out)
    print(rates)
    assert all(v > 0 for v in rates.values()), rates
    assert rates["fp32_fma"] > 8 * rates["fp64_fma"], rates
