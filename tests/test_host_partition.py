"""Host logic of the binning partition (csrc/common.cuh), compiled for the CPU
and run there: coverage of every vortex, the block bound per mode, the switch
to 1024-thread blocks and a captured launch replayed at smaller counts."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_binning_partition_host_logic(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "partition_check")
    src = os.path.join(ROOT, "tests", "host", "partition_check.cu")
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(ROOT, "paper_2102_11910_gb300", "csrc")]
    r = subprocess.run([nvcc, "-std=c++17", "-O1", *inc, src, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-2000:]
