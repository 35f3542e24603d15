"""Host logic of bench.py (CPU): the profiled figures it attaches to the
kernels stay attached across comment edits and drop out on code edits."""
import json

import bench


def test_kernel_hash_ignores_comments_not_code(tmp_path):
    a = tmp_path / "k.cuh"
    a.write_text("// a kernel\n__global__ void k(float* x) {\n  x[0] = 1.f;  // one\n}\n")
    h0 = bench.kernel_hash([str(a)])
    a.write_text("/* the same kernel,\n   documented differently */\n__global__ void k(float* x) {\n"
                 "    x[0] = 1.f;   // still one\n}\n")
    assert bench.kernel_hash([str(a)]) == h0
    a.write_text("__global__ void k(float* x) {\n  x[0] = 2.f;\n}\n")
    assert bench.kernel_hash([str(a)]) != h0


def test_profiled_traffic_only_for_the_captured_code_and_shape(tmp_path, monkeypatch):
    """bench.py reports a committed DRAM-traffic figure only while the kernels'
    code hash and the tuned work-item length are those of the capture: a
    stale summary shows up as null rather than as a number."""
    f = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    f.write_text(json.dumps({"kernel_hash": bench.kernel_hash(), "item_len": 3584,
                             "dram_bytes_per_launch": 123456789}))
    assert bench.profiled_traffic(3584) == 123456789.0
    assert bench.profiled_traffic(896) is None
    f.write_text(json.dumps({"kernel_hash": "0" * 16, "item_len": 3584, "dram_bytes_per_launch": 1}))
    assert bench.profiled_traffic(3584) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.json"))
    assert bench.profiled_traffic(3584) is None
