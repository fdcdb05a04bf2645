"""Failure detection without a GPU fault: the bounded mbarrier wait the tcgen05
kernels use returns an error status (false) when nothing arrives, instead of
spinning forever, and returns true when the arrival happens."""
import os
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_mbarrier_wait_gives_up():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "bounded_wait")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                        os.path.join(HERE, "cuda", "bounded_wait.cu"), "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "never-arrived wait returned 0, arrived wait returned 1" in r.stdout
