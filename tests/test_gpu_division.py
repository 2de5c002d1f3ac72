"""The natural cubic spline divides by 40 (Sec. IV-B.1: weights -3, 23, 23, -3
over 40).  The kernels use their own correctly rounded division by the constant
(Markstein's residual correction, an exact scaled path for tiny numerators and
an integer path for subnormal quotients) instead of a general division; this
test compiles a small checker against the library's device header and compares
it with CUDA's IEEE division __fdiv_rn on every one of the 2^32 float inputs."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.gpu
def test_div40_matches_ieee_division_on_every_float(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "div40")
    src = os.path.join(HERE, "gpu_checks", "div40_exhaustive.cu")
    subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-O3", "--fmad=false", "-std=c++17",
                    f"-I{ROOT}/include", f"-I{ROOT}/paper_2312_05492_gb300/csrc", src, "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches=0" in r.stdout
