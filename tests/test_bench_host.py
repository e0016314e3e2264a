"""Host logic of the benchmark (no GPU): the committed FP32 op tally equals a fresh
tally of the formula table, the roofline numerator is assembled from it, the kernel
source hash ignores comments but not code, and a DRAM-traffic record counts only
while the hashed kernel sources are the ones it was captured on."""
import json
import os

import bench
from paper_2603_00280_gb300 import opcounts


def test_committed_tally_matches_the_formula_table():
    fresh = opcounts.tally()
    committed = opcounts.load()
    assert fresh["ops_per_extinction_evaluation"] == committed["ops_per_extinction_evaluation"]
    assert fresh["ops_per_vertex_shading"] == committed["ops_per_vertex_shading"]
    assert fresh["per_function"] == committed["per_function"]
    f = fresh["per_function"]
    # the totals are sums of the per-formula steps; every step carries a count, or None
    # where it names another formula that the tally adds (the vertex's field fetch)
    for name, steps in opcounts.FORMULAS.items():
        assert steps and all(c is None or (isinstance(c, int) and c >= 0) for _, c in steps), name
    assert f["vertex_setup"] == sum(c for _, c in opcounts.FORMULAS["vertex_setup"] if c) + f["field_fetch"]
    assert fresh["ops_per_extinction_evaluation"] == f["field_fetch"] + f["extinction"] + f["tracking_step"]
    assert bench.opcounts() == (fresh["ops_per_extinction_evaluation"], fresh["ops_per_vertex_shading"], 64)


def test_roofline_numerator_counts_every_tentative_collision_and_vertex():
    per_eval, per_vertex, _ = bench.opcounts()
    st = {"vertices": 10, "null_collisions": 7, "shadow_steps": 5}
    assert bench.evaluations(st) == 22
    assert bench.algorithmic_ops(st) == per_eval * 22 + per_vertex * 10


def test_source_hash_ignores_comments_but_not_code():
    a = "int f(int x) {  // a note\n  return x + 1; /* block\n comment */\n}\n"
    b = "int f(int x) {\n\n  return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments(a) != bench.strip_comments(c)
    for rel in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(bench.ROOT, rel)), rel


def test_traffic_record_counts_only_for_the_captured_sources(monkeypatch):
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for name, e in t.items():
        assert e["dram_bytes_per_launch"] == e["dram_read_bytes"] + e["dram_write_bytes"], name
        assert "ncu" in e["command"] and "--clock-control none" in e["command"], name
        monkeypatch.setattr(bench, "kernel_source_hash", lambda h=e["source_hash"]: h)
        assert bench.measured_traffic(name) == e["dram_bytes_per_launch"]
        monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 12)
        assert bench.measured_traffic(name) is None
    assert bench.measured_traffic("no such workload") is None
