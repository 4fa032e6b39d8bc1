"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU and prints one JSON line on the sweep's metric and config."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--quick", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GFLOP/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    args = type("A", (), {"lo": bench.LO, "hi": bench.HI, "quick": True})()
    assert d["config"] == bench.sweep_config(args, 1)
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]


def test_reference_budget_bounds_the_run():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reference_budget(8) == 1 << 21
    assert bench.reference_budget(53) == 1 << 17
    # every step covers each small size and exactly one larger size in turn
    import paper_1203_4938_b300.inputs as I
    sizes = I.sweep_sizes(bench.TOTAL_LOG2, bench.LO, bench.HI)
    large = [t for t in sizes if t[1] > (1 << 17)]
    assert len(large) == 7


def test_traffic_hash_follows_code_not_comments():
    """The DRAM-traffic table stays valid across comment edits of the kernel
    sources and is invalidated by any code change."""
    import bench
    base = {f: "// header\nint f(int x) { /* twice */ return 2 * x; }  // done\nconst char* s = \"a // b\";\n"
            for f in bench.TRAFFIC_SOURCES}
    h0 = bench.traffic_sources_sha(lambda f: base[f])
    edited = dict(base)
    first = bench.TRAFFIC_SOURCES[0]
    edited[first] = "// new header\n\nint f(int x) {   return 2 * x; }\nconst char* s = \"a // b\";   // note\n"
    assert bench.traffic_sources_sha(lambda f: edited[f]) == h0
    changed = dict(base)
    changed[first] = base[first].replace("2 * x", "3 * x")
    assert bench.traffic_sources_sha(lambda f: changed[f]) != h0
    inside_string = dict(base)
    inside_string[first] = base[first].replace('"a // b"', '"a // c"')
    assert bench.traffic_sources_sha(lambda f: inside_string[f]) != h0
