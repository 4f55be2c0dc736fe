"""The integer-operation FP64 -> FP32 conversion and split and the
double-single product difference used by the filter's start pass
(efe_convert.cuh), over 2^28 hashed bit patterns: the conversion against the
hardware's (round to nearest even with exact ties, binary32 subnormals and
overflow, zero, inf and NaN), the split (hi the hardware's rounding at every
pattern, hi + lo within 2^-45 of x where both are binary32 normals), and
a b - c d against FP64 at cancellations down to 2^-20.  Compiled and run as
a standalone CUDA program."""
import os
import re
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2607_06848_gb300", "csrc")


def test_conversions_match_the_hardware(tmp_path):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    assert nvcc, "nvcc not found"
    exe = str(tmp_path / "convert_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-I" + CSRC,
                    os.path.join(HERE, "cuda", "convert_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    m = re.search(r"checked (\d+) f64_to_f32_rn (\d+) f64_split (\d+) ds_mul_sub (\d+)", out)
    assert m, out
    assert int(m.group(1)) == 1 << 28
    assert (int(m.group(2)), int(m.group(3)), int(m.group(4))) == (0, 0, 0), out
