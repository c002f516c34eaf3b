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


def test_algorithmic_bytes_follow_the_stated_units():
    """The roofline numerators: the streaming pass reads the frame once and
    writes the uint32 map and the 1-bit mask; the box statistics read the
    frame once; the measurement reads each segment's box (pixel and map) and
    each source's aperture window of side 2 r_max + 3."""
    import numpy as np
    import synth
    b = load_bench(ROOT)
    cfg = synth.CONFIGS["dense_12288x12304_u16"]
    npix = 12288 * 12304
    assert b.algorithmic_bytes("threshold", cfg, None) == npix * 6 + npix // 8 == 926_048_256
    assert b.algorithmic_bytes("box_stats", cfg, None) == npix * 2
    cat = {"xmin": np.array([10, 0]), "xmax": np.array([12, 4]), "ymin": np.array([5, 7]), "ymax": np.array([8, 7]),
           "npix": np.array([9, 5])}
    side = int(2 * max(cfg.radii) + 3)
    assert b.algorithmic_bytes("measure", cfg, cat) == (3 * 4 + 5 * 1) * (4 + 2) + 2 * side * side * 2
    assert b.algorithmic_bytes("label_tiles", cfg, cat) == (9 + 5) * 8
    f32 = synth.CONFIGS["plain_1024x1024_f32"]
    assert b.algorithmic_bytes("threshold", f32, None) == 1024 * 1024 * 8 + 1024 * 1024 // 8
    assert b.algorithmic_bytes("mesh_spline", cfg, None) is None
