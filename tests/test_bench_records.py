"""The DRAM-traffic record behind the bench's roofline is tied to the code it
was captured from: bench.source_hash ignores comments and whitespace but
changes with any code token, and traffic_record returns the committed
record only while the kernel source's code hash matches (CPU only)."""
import json
import os

import bench

SRC = os.path.join(bench.ROOT, "paper_1608_06473_gb300", "csrc", "cell.cu")


def test_source_hash_ignores_comments_but_not_code(tmp_path):
    code = "int f(int a) {\n  return a + 1;  // one more\n}\n"
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text(code)
    b.write_text("/* a block\n comment */\n" + code.replace("// one more", "// another note") + "\n\n")
    c.write_text(code.replace("a + 1", "a + 2"))
    assert bench.source_hash(str(a)) == bench.source_hash(str(b))
    assert bench.source_hash(str(a)) != bench.source_hash(str(c))


def test_committed_traffic_record_matches_the_current_kernel_source():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.txt")))["lsqp_node_smooth_f64@shell3840_N64"]
    assert rec["code_sha256_16"] == bench.source_hash(SRC)
    assert bench.traffic_record("lsqp_node_smooth_f64", "shell3840_N64") == rec["dram_bytes_per_sweep"]
    # 4 colour launches x 2 (3840 cells against the captured 1920)
    assert rec["dram_bytes_per_sweep"] == rec["captured_launch_bytes"] * rec["scale"] and rec["scale"] == 8.0


def test_unknown_record_is_none():
    assert bench.traffic_record("no_such_kernel", "shell3840_N64") is None
