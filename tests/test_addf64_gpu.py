"""The FP64 sum of two FP32 terms that mixed plans use for Phi = I1 + I2
(add_f32_f64: TwoSum in FP32, then the remainder added to the FP64 bit
pattern) equals the FP64 addition of the widened terms bit for bit, on 2^27
random and structured pairs (tests/cuda/addf64_check.cu)."""

import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_add_f32_f64_equals_the_fp64_addition(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "addf64_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I" + os.path.join(ROOT, "paper_1409_2014_gb300", "csrc"), "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "cuda", "addf64_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("OK 134217728"), r.stdout
