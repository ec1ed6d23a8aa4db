"""Host-side checks of the 3-centre kernels' shared-memory plans and task lists.

Compiles tests/smem_plans_check.cu against the kernel sources with nvcc (no GPU
needed) and runs it: the regions live during and after the primitive loop are
disjoint and inside the plan for every class and plan kind, and the task lists
of a synthetic shell set hold every task once, correctly marked, in a group
whose slices cover it, shape by shape.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_shared_memory_plans_and_task_lists(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "smem_plans_check")
    cmd = [nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2407_19614_gb300", "csrc"),
           "-o", exe, os.path.join(ROOT, "tests", "smem_plans_check.cu"), "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout[-3000:]
