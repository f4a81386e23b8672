"""The launch planning of the library's host code, on the CPU: builds
tests/host_plan_rules.cu (host code only, no CUDA calls) with nvcc and runs
it.  It checks, for every n and instance kind, that the chosen plan holds n,
fits shared memory, is compiled into the library and follows the stated
preferences (the products form for int8 and int16 flows wherever it is
compiled and fits, unless the dot products are asked for, and nowhere
else; 256 threads with many slots only when the walks fill two CTAs per SM,
and then two CTAs fit an SM)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_plan_rules_hold_for_every_n(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "host_plan_rules")
    build = subprocess.run(
        [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
         "-I", os.path.join(HERE, "..", "include"), os.path.join(HERE, "host_plan_rules.cu"),
         "-o", exe],
        capture_output=True, text=True, timeout=600)
    assert build.returncode == 0, build.stderr[-2000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and run.stdout.strip().endswith("ok"), run.stdout[-2000:]
