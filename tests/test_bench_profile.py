"""bench.py reads the committed ncu summary of the flip kernel (DRAM bytes per
colour pass, issue utilisation) only while the summary was taken on the current
kernel source: a changed kernel gives null, never a stale figure."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture()
def bench_copy(tmp_path, monkeypatch):
    """bench.py's profile readers pointed at a copy of the repository's
    profiles/ and kernel sources."""
    import bench
    for d in ("profiles", os.path.join("paper_1411_0127_gb300", "csrc")):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return bench, tmp_path


def test_committed_summary_matches_the_current_source(bench_copy):
    bench, _ = bench_copy
    t = bench.traffic_from_profile("mt19937")
    assert t is not None and 5e8 < t < 1e9           # about 650 MB per colour pass at L = 1024
    iss = bench.issue_from_profile("mt19937")
    assert iss is not None and 0 < iss["issue_active"] <= 1
    assert iss["warp_instructions_per_32_attempts"] > 17   # at least the algorithmic ops


@pytest.mark.parametrize("name", ["isg_flip_fast.cu", "isg_stream.cuh", "isg_common.cuh"])
def test_a_changed_kernel_source_voids_the_figures(bench_copy, name):
    bench, root = bench_copy
    p = root / "paper_1411_0127_gb300" / "csrc" / name
    p.write_text(p.read_text() + "\n// changed\n")
    assert bench.traffic_from_profile("mt19937") is None
    assert bench.issue_from_profile("mt19937") is None


def test_missing_summary_gives_null(bench_copy):
    bench, _ = bench_copy
    assert bench.traffic_from_profile("minstd") is None
