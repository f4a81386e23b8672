"""Tensor cores against the integer dot-product units on the contraction of
phase X (the dot products of Eq. 2 for the pairs touching the move).

tests/probe_phase_x_mma.cu computes, per tabu iteration, the four length-2n
matrix-vector products of phase X with dp4a and with mma.sync (f16 inputs,
f32 accumulation, exact for int8 values) and times both.  This test builds
and runs it, checks that the two forms agree exactly, and prints the
per-iteration times (run with -s to see them); it asserts nothing about
speed.  The walk kernels use the dp4a form, or products maintained by a
rank-2 update (int8 and int16 flows, wherever they fit shared memory).
"""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is available")
    nvcc = _nvcc()
    if nvcc is None:
        pytest.fail("nvcc is needed to build the probe")
    exe = str(tmp_path_factory.mktemp("probe") / "probe_phase_x_mma")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        os.path.join(HERE, "probe_phase_x_mma.cu"), "-o", exe],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


@pytest.mark.parametrize("n", [50, 100, 128])
def test_dp4a_and_mma_forms_agree(probe, n):
    r = subprocess.run([probe, str(n), "2000", "152"], capture_output=True, text=True,
                       timeout=300)
    print(r.stdout.strip())
    assert r.returncode == 0, r.stdout + r.stderr
    assert "equal=1" in r.stdout
