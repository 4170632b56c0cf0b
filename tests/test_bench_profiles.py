"""The benchmark takes a kernel's DRAM traffic from its committed ncu summary
only while the kernel's source still matches the hash recorded there."""
import hashlib
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_every_summary_gives_its_command_and_source():
    """Each summary states the ncu command (clocks left alone) and, where it
    records a traffic figure, the file and hash of the kernel's source."""
    for name in os.listdir(PROFILES):
        text = open(os.path.join(PROFILES, name)).read()
        assert "ncu " in text and "--clock-control none" in text, name
        if "traffic_bytes_per_launch" in text:
            m = re.search(r"^source: (\S+) sha256\[:16\] ([0-9a-f]{16})$", text, re.M)
            assert m and os.path.exists(os.path.join(ROOT, m.group(1))), name


def test_traffic_is_read_only_for_an_unchanged_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    digest = hashlib.sha256(b"kernel v1\n").hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k.md").write_text(
        f"traffic_bytes_per_launch: 1234\nsource: k.cu sha256[:16] {digest}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("k.md", "traffic_bytes_per_launch") == 1234
    src.write_text("kernel v2\n")
    assert bench.profiled_traffic("k.md", "traffic_bytes_per_launch") is None
    assert bench.profiled_traffic("missing.md", "traffic_bytes_per_launch") is None
