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


def test_reference_arm_prints_one_line():
    """`bench.py --impl reference` walks the benchmark surface with the oracle
    on the host's cores and prints the contract's JSON line."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], cwd=root, capture_output=True, text=True,
                         timeout=600, check=True).stdout.strip().splitlines()
    assert len(out) == 1
    d = json.loads(out[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_line_moves_summary():
    N = 64
    t = [0, 0] + [1000 * (l + 1) for l in range(2, N // 2 + 1)]   # lines 0 and 1 never walk
    r = bench.line_moves_summary(t, N)
    assert r["lines_walked"] == N // 2 - 1
    assert r["max"] == 33000 and r["argmax_l"] == N // 2
    assert r["paper_lines"] == {"8": 9000, "16": 17000, "24": 25000, "32": 33000}
    assert sum(r["log2_histogram"].values()) == r["lines_walked"]
    assert r["log2_histogram"]["2^11"] == 2                        # 3000 and 4000 lie in [2048, 4096)
    assert r["log2_histogram"]["2^14"] == 16                       # 17000 .. 32000
