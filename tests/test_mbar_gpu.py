"""The bounded mbarrier wait and the asynchronous copies the prefetching row
passes use (common.cuh): an expired wait returns false after its limit (the
status path, exercised with a phase that nothing completes; no fault, no
hang), an arrival and a bulk copy complete their phases, bulk and cp.async
copies deliver their data, and a CTA whose wait expired records
DSNU_ETIMEOUT and returns without writing (cta_timed_out)."""

import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounded_mbarrier_wait_and_async_copies(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "mbar_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I" + os.path.join(ROOT, "paper_1409_2014_gb300", "csrc"), "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "cuda", "mbar_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("OK"), r.stdout
