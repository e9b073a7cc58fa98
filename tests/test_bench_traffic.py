"""bench.py reports recorded DRAM traffic only for the kernel source it was taken on.

The source hash ignores comments and blank lines, so documentation edits keep a
recorded figure; any change to the code makes it null until re-taken.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _tree(tmp_path, src):
    d = tmp_path / "paper_2512_01055_gb300" / "csrc"
    d.mkdir(parents=True)
    (d / "tc_split.cu").write_text(src)
    (d / "tc_ptx.cuh").write_text("// shared helpers\n#pragma once\n")
    (tmp_path / "profiles").mkdir()
    return tmp_path


def test_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    base = "int f(int x) {\n  return x + 1;  // add one\n}\n"
    monkeypatch.setattr(bench, "ROOT", str(_tree(tmp_path, base)))
    h0 = bench.kernel_source_hash("split")
    p = tmp_path / "paper_2512_01055_gb300" / "csrc" / "tc_split.cu"
    p.write_text("/* a header\n   comment */\n\nint f(int x) {\n  return x + 1;  // one more\n}\n")
    assert bench.kernel_source_hash("split") == h0
    p.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.kernel_source_hash("split") != h0
    p.write_text(base)
    (tmp_path / "paper_2512_01055_gb300" / "csrc" / "tc_ptx.cuh").write_text("#pragma once\nint h();\n")
    assert bench.kernel_source_hash("split") != h0          # the shared helpers count too


def test_recorded_traffic_follows_the_hash(tmp_path, monkeypatch):
    root = _tree(tmp_path, "int g() { return 0; }\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec = {"tc_wterm_kernel:w": {"dram_bytes_per_launch": 123, "source_sha": bench.kernel_source_hash("split")}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("tc_wterm_kernel", "w", "split") == 123
    (root / "paper_2512_01055_gb300" / "csrc" / "tc_split.cu").write_text("int g() { return 1; }\n")
    assert bench.recorded_traffic("tc_wterm_kernel", "w", "split") is None

