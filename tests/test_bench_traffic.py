"""The DRAM traffic that bench.py reports beside the roofline comes from a
committed ncu summary, and only while the measured kernel's sources are the
ones the counters were taken on: any change to them must turn the figure
into null rather than report stale counters."""
import importlib.util
import json
import os
import shutil

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
    assert "k_detect_tile" in d                      # the dominant kernel
    for kernel, e in d.items():
        assert e["read"] + e["write"] == e["dram_bytes_per_launch"]
        assert os.path.exists(os.path.join(ROOT, e["summary"]))
        # either the counters of the current sources, or null once they changed
        assert b.kernel_traffic(kernel, e["workload"]) in (float(e["dram_bytes_per_launch"]), None), kernel


def test_traffic_turns_null_when_a_source_changes(tmp_path):
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    kernel, e = next(iter(d.items()))
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    for src in e["sources"]:
        os.makedirs(os.path.dirname(tmp_path / src), exist_ok=True)
        shutil.copy(os.path.join(ROOT, src), tmp_path / src)
    b = load_bench(str(tmp_path))
    assert b.kernel_traffic(kernel, e["workload"]) == float(e["dram_bytes_per_launch"])
    assert b.kernel_traffic(kernel, "another_workload") is None
    with open(tmp_path / e["sources"][0], "a") as f:
        f.write("\n// changed\n")
    assert b.kernel_traffic(kernel, e["workload"]) is None
    assert b.kernel_traffic("no_such_kernel", e["workload"]) is None
