"""CPU tests of bench.py's host logic: the traffic record is keyed on the
kernel's code (comments ignored) and on the kernel's name."""
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


def test_traffic_record_needs_the_recorded_kernel():
    src = os.path.join(ROOT, "paper_2012_08141_gb300", "csrc", "sg_sweep.cu")
    assert bench.traffic_record(src, "k_not_a_kernel<false,false,true>") is None
    v = bench.traffic_record(src, bench.KERNEL_NAMES[3])
    assert v is None or v > 0
