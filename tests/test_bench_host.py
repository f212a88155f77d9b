"""Host-side arithmetic of bench.py on hand-computed values (no GPU): the
harmonic mean, the rank combination, the byte models behind the roofline
figures, and the rule that the recorded DRAM traffic is reported only while
the hub sweep kernel's source is the one that was measured."""
from __future__ import annotations

import os

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
    # 3n/4 + 4 per probed vertex + 8 per written vertex
    assert bench.hub_sweep_bytes(1024, 300, 20) == 768 + 1200 + 160
    assert bench.hub_sweep_bytes(1024, 300, 20, 4) == 768 + 1200 + 80
    # 1e9 edges at 1000 GB/s with 1e10 bytes per traversal: 100 GTEPS
    assert bench.roofline_teps(1e9, 1000.0, 1e10) == pytest.approx(1e11)
    # batched: k = 128 (W = 2), n = 1000, two layers examining 10 and 30
    # entries: (4 + 16) * 40 + 2 * 3 * 16 * 1000 + 128 * 1000
    layers = [{"examined": 10}, {"examined": 30}]
    assert bench.batch_bytes(1000, 128, layers) == 20 * 40 + 96000 + 128000


def _tree_copy(tmp_path, profile_text, src_edit=None):
    os.makedirs(tmp_path / "profiles", exist_ok=True)
    os.makedirs(tmp_path / "paper_1704_02259_gb300" / "csrc", exist_ok=True)
    (tmp_path / "profiles" / "bu_hubc_stream_kernel_rmat24.md").write_text(profile_text)
    src = open(os.path.join(HERE, "paper_1704_02259_gb300", "csrc", "bfs.cu")).read()
    if src_edit:
        src = src_edit(src)
    (tmp_path / "paper_1704_02259_gb300" / "csrc" / "bfs.cu").write_text(src)


def test_traffic_reported_only_for_the_measured_kernel(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha1("bu_hubc_stream_kernel")
    assert sha
    text = ("# capture\n\ncapture_scale: 24\ntraffic_first_sweep_bytes: 400\n"
            f"traffic_later_sweep_bytes: 100\nkernel_source_sha1: {sha}\n")
    _tree_copy(tmp_path, text)
    monkeypatch.setattr(bench, "HERE", str(tmp_path))
    # 3 launches, 1 of them a first sweep, at scale 26: (400 + 2 * 100) / 3 * 4
    assert bench.measured_traffic("bu_hubc_stream_kernel", 26, 16, 3, 1) == pytest.approx(800.0)
    assert bench.measured_traffic("bu_hubc_stream_kernel", 24, 16, 1, 1) == pytest.approx(400.0)
    assert bench.measured_traffic("bu_hubc_stream_kernel", 26, 32, 3, 1) is None
    assert bench.measured_traffic("bu_hubc_kernel", 26, 16, 3, 1) is None  # no summary
    # the kernel's source changed by one character inside the hashed text
    marker = bench.KERNEL_TEXT["bu_hubc_stream_kernel"][0]

    def edit(src):
        k = src.find(marker) + len(marker) + 5
        return src[:k] + "#" + src[k + 1:]
    _tree_copy(tmp_path, text, edit)
    assert bench.measured_traffic("bu_hubc_stream_kernel", 26, 16, 3, 1) is None


def test_committed_traffic_summaries_match_their_kernels():
    # every committed sweep summary carries the hash of the current source
    for name in bench.KERNEL_TEXT:
        path = os.path.join(HERE, "profiles", f"{name}_rmat24.md")
        if os.path.exists(path):
            assert bench.measured_traffic(name, 24, 16, 2, 1) is not None, name


def test_table3_constant_matches_the_fixture():
    rows = []
    with open(os.path.join(HERE, "tests", "golden",
                           "table3_bu_edges_per_visited_scale18_ef16.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(float(line.split()[1]))
    assert rows == [float(x) for x in bench.TABLE3_PAPER]
