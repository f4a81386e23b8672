"""The benchmark's roofline arithmetic and its use of the committed ncu
figures, on the CPU (bench.py imported, nothing launched)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_unit_bytes_per_walk_iteration():
    """T(2w + 2) + (1 symmetric | 2 asymmetric) n^2 (eF + eP): every delta
    read and written, a 2-byte tabu stamp read per pair, and the rows (and
    columns) of F and P read for the recomputed pairs.  n = 50 asymmetric,
    int32 deltas, int8 F and P: 1225 * 10 + 2 * 2500 * 2 = 22250 bytes."""
    assert bench.unit_bytes(50, 4, 1, 1, sym=False) == 22250
    assert bench.unit_bytes(50, 4, 1, 1, sym=True) == 1225 * 10 + 2500 * 2
    # int64 deltas, int16 flows: the lognormal batch instances
    assert bench.unit_bytes(100, 8, 2, 1, sym=False) == 4950 * 18 + 2 * 10000 * 3


def test_derived_peaks():
    # 128 B per clock per SM, 152 SMs at 2070 MHz
    assert bench.smem_peak_gbs(152, 2070.0) == pytest.approx(40273.92)
    # four schedulers, one warp instruction each per clock
    assert bench.issue_peak(152, 2070.0) == pytest.approx(4 * 152 * 2.07e9)


def test_rooflines_with_and_without_committed_figures():
    figs = {"warp_insts_per_unit": 3000.0, "dram_bytes_per_launch": 1.0e5}
    roof, issue = bench.rooflines(2.0e10, 1.0e6, 0.01, 152, 2070.0, figs, "k")
    assert roof["achieved"] == pytest.approx(2.0e10 / 0.01 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / bench.smem_peak_gbs(152, 2070.0))
    assert roof["traffic"] == 1.0e5
    assert issue["achieved"] == pytest.approx(3000.0 * 1.0e6 / 0.01)
    assert issue["frac"] == pytest.approx(issue["achieved"] / bench.issue_peak(152, 2070.0))
    roof, issue = bench.rooflines(2.0e10, 1.0e6, 0.01, 152, 2070.0, {}, "k")
    assert roof["traffic"] is None and issue is None


@pytest.mark.parametrize("name", ["batch_kernel_batch512", "walk_kernel_asym50",
                                  "walk_kernel_grid100"])
def test_committed_profile_figures(name):
    """A summary under profiles/ gives its figures under its own key and
    nothing under another; while its key is the current sources' (kernels
    and plan rules), the bench reads a positive warp-instruction count from
    it (otherwise it reports no issue bound, and this test says so)."""
    import re
    text = open(os.path.join(ROOT, "profiles", name + ".md")).read()
    key = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text).group(1)
    assert bench.profile_figures(name, key).get("warp_insts_per_unit", 0) > 0
    assert bench.profile_figures(name, "0" * 16) == {}
    if key != bench.kernel_source_hash():
        pytest.skip(f"{name} was taken on other kernel sources ({key})")


def test_source_hash_ignores_comments(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2307_11248_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ("a.cuh",))
    (csrc / "a.cuh").write_text("int f() { return 1; }\n")
    h1 = bench.kernel_source_hash()
    (csrc / "a.cuh").write_text("// a comment\n\nint f() { return 1; }  // another\n")
    assert bench.kernel_source_hash() == h1
    (csrc / "a.cuh").write_text("int f() { return 2; }\n")
    assert bench.kernel_source_hash() != h1
