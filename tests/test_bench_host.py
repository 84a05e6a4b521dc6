"""Host logic of bench.py that needs no GPU: the traffic figure is only used
while the walker source it was measured on is unchanged."""
import os

import bench


def test_traffic_figure_requires_matching_kernel(tmp_path, monkeypatch):
    f = tmp_path / "traffic.txt"
    h = bench.kernel_source_hash()
    f.write_text(f"# test\nkernel_source_sha256: {h}\nmoves_per_line: 4194304\nmapping: 32\n"
                 f"dram_bytes_per_launch: 123456\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.walker_traffic(4194304, 32) == 123456
    assert bench.walker_traffic(65536, 32) is None          # another launch shape
    assert bench.walker_traffic(4194304, 8) is None
    f.write_text(f.read_text().replace(h, "0" * 16))
    assert bench.walker_traffic(4194304, 32) is None          # kernel changed since


def test_kernel_hash_is_stable():
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert len(bench.kernel_source_hash()) == 16
