"""Host logic of bench.py's measurement: the byte ledger of a sort (the passes it
makes and the minimum one-level ledger, closed forms per key) and the gate that
uses ncu traffic figures only for the sources they were captured on."""
import json
import os

import bench


def test_ledger_closed_forms_int32_keys_only():
    n = 1 << 20
    # every key split once more in the bucket phase, no deeper repartition
    led = bench.pipeline_ledger(n, 4, 0, n, n, ms=1.0, peak=1000.0)
    # top classify k+2, scatter 2k+2, bucket-phase split (k+2) + (2k+2), leaf 2k: 40 B for k = 4
    assert led["actual_bytes"] == 40 * n
    assert led["min_bytes"] == 20 * n                # classify k, scatter 2k, sort 2k
    assert abs(led["actual_gbs"] - 40 * n / 1e-3 / 1e9) < 0.1
    assert led["comparisons"] == round(n * 20)        # n lg n


def test_ledger_payload_and_repartition():
    n, k, v = 1 << 16, 8, 4
    base = bench.pipeline_ledger(n, k, v, 0, 0, 1.0, 1.0)
    more = bench.pipeline_ledger(n, k, v, 0, 1000, 1.0, 1.0)
    assert more["actual_bytes"] - base["actual_bytes"] == 1000 * (3 * k + 2 * v)
    assert base["min_bytes"] == n * (k + 4 * (k + v))


def test_traffic_used_only_for_its_sources(tmp_path, monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "kernel_traffic_i32.json")
    with open(path) as f:
        t = json.load(f)
    per = t["dram_bytes_per_key"]["k_leaf"]
    monkeypatch.setattr(bench, "cuda_source_sha", lambda: t["source_sha"])
    assert bench.measured_traffic("k_leaf", "i32", 1000) == int(per * 1000)
    with open(os.path.join(bench.ROOT, "profiles", "kernel_traffic_f64.json")) as f:
        t64 = json.load(f)
    monkeypatch.setattr(bench, "cuda_source_sha", lambda: t64["source_sha"])
    assert bench.measured_traffic("k_leaf", "f64", 1000) == int(t64["dram_bytes_per_key"]["k_leaf"] * 1000)
    monkeypatch.setattr(bench, "cuda_source_sha", lambda: "0" * 16)
    assert bench.measured_traffic("k_leaf", "i32", 1000) is None
    assert bench.measured_traffic("k_leaf", "f64", 1000) is None
    assert bench.measured_traffic("k_leaf", "u64", 1000) is None      # no capture for uint64


def test_split_merge_ledger():
    """The split + merge SqDet: one gather pass, then ceil(log2 p) pairwise merge passes,
    each reading and writing every key and payload."""
    n = 1 << 20
    assert bench.algorithmic_bytes("k_det_gather", n, 4, 0, 0) == 8 * n
    assert bench.algorithmic_bytes("k_det_merge", n, 4, 0, 0, 0, 1024) == 8 * n * 10
    assert bench.algorithmic_bytes("k_det_merge", n, 8, 4, 0, 0, 1000) == 24 * n * 10
    assert bench.algorithmic_bytes("k_det_merge", n, 4, 0, 0, 0, 2) == 8 * n


def test_secondary_bound_used_only_for_its_sources(monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "kernel_traffic_i32.json")
    with open(path) as f:
        t = json.load(f)
    monkeypatch.setattr(bench, "cuda_source_sha", lambda: t["source_sha"])
    sec = bench.measured_pipe("k_leaf", "i32")
    if "pipes" in t:
        assert sec is not None and 0 < sec["alu_pipe_pct"] <= 100 and "ncu" in sec["source"]
    monkeypatch.setattr(bench, "cuda_source_sha", lambda: "0" * 16)
    assert bench.measured_pipe("k_leaf", "i32") is None
    assert bench.measured_pipe("k_leaf", "f64") is None
