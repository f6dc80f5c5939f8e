"""Launch plans of the tensor-core kernels, checked on the host: the header's
plan functions are compiled into a small host program (tc_plan_check.cu) that
tests them against the alignment, shared-memory and tensor-memory rules the
kernels rely on, for every channel pair the network's convolutions accept."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tensor_core_launch_plans(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "tc_plan_check")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                    os.path.join(HERE, "tc_plan_check.cu")], check=True, capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "40 channel pairs checked, 0 failures" in r.stdout
