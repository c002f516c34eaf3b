"""The DRAM traffic that bench.py reports beside the roofline comes from a
committed ncu summary, and only while the measured kernel's sources are the
ones the counters were taken on: any change to them must turn the figure
into null rather than report stale counters."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench(root):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.ROOT = root
    return b


def test_committed_traffic_is_well_formed():
    b = load_bench(ROOT)
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert "k_stream" in d                           # the dominant kernel
    for kernel, e in d.items():
        assert e["read"] + e["write"] == e["dram_bytes_per_launch"]
        assert os.path.exists(os.path.join(ROOT, e["summary"]))
        # either the counters of the current sources, or null once they changed
        assert b.kernel_traffic(kernel, e["workload"]) in (float(e["dram_bytes_per_launch"]), None), kernel


def test_traffic_turns_null_when_a_source_changes(tmp_path):
    import hashlib
    src = tmp_path / "csrc" / "k_x.cu"
    os.makedirs(src.parent)
    src.write_text("__global__ void k_x() {}\n")
    entry = {"workload": "w", "dram_bytes_per_launch": 3, "read": 2, "write": 1, "sources": ["csrc/k_x.cu"],
             "sources_sha1": hashlib.sha1(src.read_bytes()).hexdigest(), "summary": "profiles/x.md"}
    os.makedirs(tmp_path / "profiles")
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"k_x": entry}))
    b = load_bench(str(tmp_path))
    assert b.kernel_traffic("k_x", "w") == 3.0
    assert b.kernel_traffic("k_x", "another_workload") is None
    assert b.kernel_traffic("k_y", "w") is None
    src.write_text("__global__ void k_x() { /* changed */ }\n")
    assert b.kernel_traffic("k_x", "w") is None
