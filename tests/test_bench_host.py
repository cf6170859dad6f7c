"""Host-side pieces of bench.py (no GPU): the traffic record's key ignores
comment edits but not code edits, the committed record parses, and the
replica rate of a single process is units over seconds."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_source_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2308_10674_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("epie_fft.cuh", "epie_cluster.cuh", "epie_fused_256.cu"):
        shutil.copy(os.path.join(ROOT, "paper_2308_10674_gb300", "csrc", f), csrc / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.source_hash()
    p = csrc / "epie_fused_256.cu"
    p.write_text(p.read_text() + "\n// a new comment line\n\n")
    assert bench.source_hash() == h0
    p.write_text(p.read_text().replace("constexpr int CP", "constexpr  int CP", 1))
    assert bench.source_hash() != h0


def test_committed_traffic_record_parses():
    rec = {}
    with open(os.path.join(ROOT, "profiles", "fused_256_traffic.txt")) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
    assert len(rec["source_hash"]) == 16
    assert float(rec["dram_bytes_per_frame"]) > 256 * 256 * 2


def test_replica_rate_single_process():
    value, secs = bench.replica_rate(1000, 2.0)
    assert value == pytest.approx(500.0) and secs == pytest.approx(2.0)


def test_step_kernel_names_follow_frame_side_and_tile_shape():
    assert bench.step_kernel_name(256) == "epie_fused256_kernel"
    assert bench.step_kernel_name(512) == "epie_fused512_kernel"
    assert bench.step_kernel_name(128) == "epie_fused_kernel<128,4,...>"
    assert bench.step_kernel_name(128, 1) == "epie_fused128_kernel"
    assert bench.step_kernel_name(64) == "epie_fused_kernel<64,1,...>"


def test_metric_names_the_frame_side_and_path():
    assert bench.metric_name() == bench.METRIC
    assert bench.metric_name(512) == "ePIE frame-updates/s at 512^2 px (fused path), error vs FP64 oracle"
    assert "(plain path)" in bench.metric_name(256, "plain")


def test_traffic_record_matches_the_committed_kernel():
    # the record is retaken whenever the 256^2 step kernel's code changes
    assert bench.measured_traffic() is not None
