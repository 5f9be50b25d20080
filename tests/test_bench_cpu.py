"""CPU tests of the benchmark's bookkeeping: the kernel-source hash that ties a
recorded DRAM capture to the sources it was taken of, and the lookup that
reports the capture only for those sources and that workload size."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture()
def bench(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    import bench as b
    return b


def test_source_hash_is_stable_and_covers_the_sources(bench, tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()
    # a copy of the tree with one source byte changed hashes differently
    fake = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "paper_2511_17245_gb300", "csrc"), fake / "paper_2511_17245_gb300" / "csrc")
    shutil.copytree(os.path.join(ROOT, "include"), fake / "include")
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.kernel_source_hash() == h
    with open(fake / "paper_2511_17245_gb300" / "csrc" / "sweep.cuh", "a") as fh:
        fh.write("\n")
    assert bench.kernel_source_hash() != h


def test_captured_traffic_only_for_matching_sources_and_size(bench, tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    fake = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "paper_2511_17245_gb300", "csrc"), fake / "paper_2511_17245_gb300" / "csrc")
    shutil.copytree(os.path.join(ROOT, "include"), fake / "include")
    (fake / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.captured_traffic("heat_bath", 1000, 1024) == (None, "no capture recorded")
    rec = fake / "profiles" / "dram_heat_bath_quio_sparse_wide.md"
    rec.write_text(f"x\ntraffic: dram_bytes_per_launch=123456 sweeps=1000 replicas=1024 source_hash={h}\n")
    val, src = bench.captured_traffic("heat_bath", 1000, 1024)
    assert val == 123456 and "one launch" in src
    assert bench.captured_traffic("heat_bath", 50, 1024)[0] is None
    assert bench.captured_traffic("metropolis", 1000, 1024)[0] is None
    rec.write_text("traffic: dram_bytes_per_launch=123456 sweeps=1000 replicas=1024 source_hash=0000000000000000\n")
    assert bench.captured_traffic("heat_bath", 1000, 1024) == (None, "sources changed since the capture")


def test_committed_capture_is_readable(bench):
    """The DRAM record under profiles/ parses; while it belongs to these
    sources the benchmark reports it, otherwise it reports null."""
    val, src = bench.captured_traffic("heat_bath", 1000, 1024)
    if val is None and src == "sources changed since the capture":
        pytest.skip("kernel sources changed since the recorded capture: traffic is null until it is retaken")
    assert val is not None and val > 0, src
