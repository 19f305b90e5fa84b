"""Failure detection of the tensor-core pipeline without a GPU fault: its mbarrier waits are
bounded, a wait that nothing completes expires and is reported as a status (the library turns
it into GBXC_ETIMEOUT), and the context keeps running work (tests/cuda/bounded_wait_check.cu)."""
import json
import os
import shutil
import subprocess

import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2007_03143_gb300", "csrc")


def test_bounded_wait_expires_and_context_survives(tmp_path):
    need_gpu()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "bounded_wait_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC,
                    os.path.join(HERE, "cuda", "bounded_wait_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert r.returncode == 0, res
    assert res["timed_out"] == 1 and res["completed_seen"] == 1 and res["after"] == 64
