"""The work schedules of the tensor-core passes (raster, stream-K and the hybrid of the two):
every (unit, k-block) is processed exactly once and the fix-up reads exactly the partial slots
the kernels write.  Host-only: tests/sched_check.cu includes the schedule header the kernels
use, is compiled with nvcc and run on the CPU over ~9000 pass shapes."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_schedules_cover_every_k_block_and_match_the_fixup(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = tmp_path / "sched_check"
    src = os.path.join(ROOT, "tests", "sched_check.cu")
    inc = os.path.join(ROOT, "paper_1606_09402_gb300", "csrc")
    b = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", inc, "-o", str(exe), src],
                       capture_output=True, text=True, timeout=600)
    assert b.returncode == 0, b.stdout + b.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 failures" in r.stdout
    # the hybrid schedule is exercised (the 4.1-wave passes of the 40000 x 20000 step use it)
    assert "hybrid 0;" not in r.stdout
