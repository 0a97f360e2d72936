"""The FP64 pivot reciprocal of the coarse factorisations (csrc/rcp64.h:
the rcp.approx.ftz.f64 estimate and one Halley step) against IEEE 1/d on
2^22 random values of both signs over 600 binades: within one ulp of the
correctly rounded reciprocal, i.e. relative error below 2^-52."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1705_05783_gb300", "csrc")


def test_rcp_halley_against_ieee_division(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "rcp64_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-I", CSRC,
                    os.path.join(HERE, "rcp64_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    print(out)
    f = out.split()
    max_ulp, max_rel = int(f[1]), float(f[3])
    assert max_ulp <= 1 and max_rel < 2.0 ** -52
