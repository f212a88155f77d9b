"""Host-side arithmetic of bench.py on hand-computed values (no GPU): the
harmonic mean, the rank combination, the byte models behind the roofline
figures, and the rule that the recorded DRAM traffic is reported only while
the hub sweep kernel's source is the one that was measured."""
from __future__ import annotations

import os
import shutil

import pytest

import bench

HERE = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_harmonic_mean():
    assert bench.hmean([1.0, 2.0, 4.0]) == pytest.approx(3 / (1 + 0.5 + 0.25))
    assert bench.hmean([5.0]) == 5.0
    assert bench.hmean([]) == 0.0
    assert bench.hmean([3.0, 0.0]) == 0.0        # a zero rate is not averaged away


def test_combine_ranks():
    value, t, wall = bench.combine_ranks([[10.0, 2.0, 3.0], [30.0, 2.5, 1.0]])
    assert (value, t, wall) == (40.0, 2.5, 3.0)


def test_byte_models():
    # n = 2^10, nnz = 5000: 4*5000 + 8*1025 + 2*128 + 8*1024
    assert bench.one_sweep_bytes(1024, 5000) == 20000 + 8200 + 256 + 8192
    # n/2 + 8 per probed vertex + 8 per written vertex
    assert bench.hub_sweep_bytes(1024, 300, 20) == 512 + 2400 + 160
    # 1e9 edges at 1000 GB/s with 1e10 bytes per traversal: 100 GTEPS
    assert bench.roofline_teps(1e9, 1000.0, 1e10) == pytest.approx(1e11)


def test_traffic_reported_only_for_the_measured_kernel(tmp_path, monkeypatch):
    recorded = bench.measured_traffic(26, 16)
    assert recorded is not None and recorded > 0
    assert bench.measured_traffic(22, 16) is None      # another workload
    # a copy of the tree whose hub sweep source differs by one character
    os.makedirs(tmp_path / "profiles")
    os.makedirs(tmp_path / "paper_1704_02259_gb300" / "csrc")
    shutil.copy(os.path.join(HERE, "profiles", "bu_hub_kernel_dram_rmat26.md"),
                tmp_path / "profiles")
    src = open(os.path.join(HERE, "paper_1704_02259_gb300", "csrc", "bfs.cu")).read()
    marker = "// First pass of the two-pass bottom-up step"
    a = src.find(marker)
    assert a >= 0
    k = a + len(marker) + 10                       # inside the hashed text
    assert src[k] != "#"
    (tmp_path / "paper_1704_02259_gb300" / "csrc" / "bfs.cu").write_text(
        src[:k] + "#" + src[k + 1:])
    monkeypatch.setattr(bench, "HERE", str(tmp_path))
    assert bench.measured_traffic(26, 16) is None
    (tmp_path / "paper_1704_02259_gb300" / "csrc" / "bfs.cu").write_text(src)
    assert bench.measured_traffic(26, 16) == recorded


def test_table3_constant_matches_the_fixture():
    rows = []
    with open(os.path.join(HERE, "tests", "golden",
                           "table3_bu_edges_per_visited_scale18_ef16.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(float(line.split()[1]))
    assert rows == [float(x) for x in bench.TABLE3_PAPER]
