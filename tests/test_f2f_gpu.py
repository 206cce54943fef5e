"""The FP64 -> FP32 rounding that the forward row pass does with integer
instructions for half of its values (f32_of_f64_int, the hardware conversion
for the values it flags) equals the hardware's round-to-nearest conversion
bit for bit, on 2^27 random and structured doubles (tests/cuda/f2f_check.cu)."""

import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_f32_of_f64_int_equals_the_hardware_rounding(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "f2f_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I" + os.path.join(ROOT, "paper_1409_2014_gb300", "csrc"), "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "cuda", "f2f_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("OK 134217728"), r.stdout
