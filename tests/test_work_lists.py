"""Host-side check of the persistent kernels' work lists, no GPU: nvcc builds
tests/work_lists_check.cu (which includes the library's ibs_tc.cu) and runs it
on the CPU.  It covers the one-SM list (tc_single_items) and the two-SM pair
list (tc_pair_items) over 10 sample counts, 8 marker counts (up to 2.2 M
markers, past the 2^21-marker exact-accumulation limit) and 5 SM/cluster
counts: each upper-triangle tile covered once over the whole K range, the
split-tile list exact, no item beyond 2^21 markers."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_work_lists_cover_the_triangle(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "work_lists_check")
    build = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                            "-I", os.path.join(ROOT, "include"), "-o", exe,
                            os.path.join(ROOT, "tests", "work_lists_check.cu")],
                           capture_output=True, text=True, timeout=600)
    assert build.returncode == 0, build.stdout + build.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout[-4000:]
    assert ", 0 failures" in run.stdout and "checked 680 lists" in run.stdout, run.stdout[-2000:]
