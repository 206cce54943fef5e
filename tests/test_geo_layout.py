"""Host-only static check (no GPU) of the shared-memory layouts of the
pipeline kernels for every grid size and both precisions: sizes within the
per-CTA limit, 16-byte alignment of every asynchronous-copy target, the
mbarrier alignment and the CTAs per SM of the prefetching row passes
(tests/cuda/geo_check.cu, built with nvcc for the host)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shared_memory_layouts(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "geo_check")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "paper_1409_2014_gb300", "csrc"),
                    "-I" + os.path.join(ROOT, "include"), "-x", "cu",
                    os.path.join(ROOT, "tests", "cuda", "geo_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
