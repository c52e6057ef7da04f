"""CPU tests of bench.py's host logic: the traffic record is keyed on the
code (comments ignored) of every source that shapes the kernel's access
order, on the kernel's name and on the workload."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_sha1_ignores_comments_not_code(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("int f(int x)\n{\n    return x + 1;  // one\n}\n")
    b.write_text("/* header\n   comment */\nint f(int x)\n{\n\n    return x + 1;\n}\n// trailing\n")
    c.write_text("int f(int x)\n{\n    return x + 2;\n}\n")
    assert bench.code_sha1(str(a)) == bench.code_sha1(str(b))
    assert bench.code_sha1(str(a)) != bench.code_sha1(str(c))


def test_traffic_record_needs_the_recorded_kernel_and_sources(tmp_path):
    p = tmp_path / "traffic.json"
    rec = {"kernel": bench.KERNEL_NAMES[4], "workload": "512^3 band, 26104 leaves",
           "sources_sha1": bench.sources_sha1(4), "dram_bytes_per_launch": 123}
    p.write_text(json.dumps([rec]))
    assert bench.traffic_record(4, path=str(p)) == 123
    assert bench.traffic_record(4, "1024^3 band", path=str(p)) is None
    assert bench.traffic_record(3, path=str(p)) is None          # another kernel
    p.write_text(json.dumps([dict(rec, sources_sha1="0" * 40)]))
    assert bench.traffic_record(4, path=str(p)) is None          # a source changed since the capture
    # the region-mask / run-record source is part of the key
    assert "sg_structure.cu" in bench.KERNEL_SRCS[4] and "sg_structure.cu" in bench.KERNEL_SRCS[3]
    v = bench.traffic_record(3)
    assert v is None or v > 0
