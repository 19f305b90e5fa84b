"""The library's own device arithmetic against CUDA's float64 results and its stated bounds:
the double-float exp(-t) used by the tensor-core form's collocation (Cody-Waite reduction,
Taylor series, squarings) and the Ozaki slicing of its contractions (reconstruction within
2^-34 of the row scale, integer slices within their magnitude bounds, exact in bf16)."""
import json
import os
import shutil
import subprocess

import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2007_03143_gb300", "csrc")


def test_device_math(tmp_path):
    need_gpu()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "device_math_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC,
                    os.path.join(HERE, "cuda", "device_math_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    print(res)
    assert r.returncode == 0, res
    assert res["exp_max_rel_t_le_70"] < 1e-12
    assert res["slice_max_err"] <= 2.0 ** -34
    assert res["slice_max_units"][0] <= 64 and res["slice_max_units"][1] <= 64 and res["slice_max_units"][2] <= 64
