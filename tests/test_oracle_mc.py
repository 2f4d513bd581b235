"""Pins of the oracle's multi-core form (Section 2.4: the p sorts of step 1, and
optionally the p merges of step 5, split over threads) and of SomeSort run
alone: the multi-core form must give the single-thread oracle's outputs bit for
bit (keys, payload, splitters, tags, bucket sizes) for any thread count,
including counts that do not divide p and counts above p; SomeSort alone must
give numpy's stable argsort order."""
import numpy as np
import pytest

import oracle
from paper_1608_08648_gb300 import inputs

FIELDS = ("keys", "vals", "spl_keys", "spl_tags", "bucket_sizes")


@pytest.mark.parametrize("kt", ["i32", "u64", "f64"])
@pytest.mark.parametrize("split", ["det", "ran"])
@pytest.mark.parametrize("threads,par5", [(2, False), (3, True), (7, True), (64, True), (500, False)])
def test_multicore_equals_single_thread(kt, split, threads, par5):
    n, p, s = 100_003, 64, 4
    keys = inputs.keys("dup" if kt == "i32" else "uniform", n, kt, seed=3).numpy()
    vals = np.arange(n, dtype=np.uint32)
    a = oracle.sort(keys, kt, split, p, s, seed=5, vals=vals)
    b = oracle.sort(keys, kt, split, p, s, seed=5, vals=vals, threads=threads, par_step5=par5)
    for f in FIELDS:
        assert np.array_equal(a[f], b[f]), f
    assert a["p_used"] == b["p_used"] == p


def test_multicore_strings_and_small_input():
    keys = inputs.strings("prefix8", 20_011, seed=4).numpy()
    a = oracle.sort(keys, "s32", "ran", 16, 4, seed=2)
    b = oracle.sort(keys, "s32", "ran", 16, 4, seed=2, threads=4, par_step5=True)
    for f in ("keys", "spl_keys", "spl_tags", "bucket_sizes"):
        assert np.array_equal(a[f], b[f]), f
    small = inputs.keys("uniform", 100, "i32", seed=1).numpy()     # too small to sample: one bucket
    c = oracle.sort(small, "i32", "det", 8, 4, threads=4, par_step5=True)
    assert c["p_used"] == 1 and np.array_equal(c["keys"], np.sort(small))


@pytest.mark.parametrize("kt", ["i32", "u64", "f64"])
def test_some_sort_alone_is_the_stable_sort(kt):
    n = 50_021
    keys = inputs.keys("dup" if kt != "f64" else "gaussian", n, kt, seed=9).numpy()
    vals = np.arange(n, dtype=np.uint32)
    r = oracle.some_sort(keys, kt, vals=vals)
    perm = np.argsort(keys, kind="stable")
    assert np.array_equal(r["keys"], keys[perm])
    assert np.array_equal(r["vals"], vals[perm])


def test_bench_cpu_baseline_fields():
    import argparse

    import bench
    a = argparse.Namespace(cpu_sample=1 << 14, keys=1 << 20, dist="uniform", dtype="i32", seed=1, p=16, s=4,
                           split="ran")
    cb = bench.cpu_baseline(a, "i32", 16)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] > 0
    assert "median of 3" in cb["sample"]
    one = bench.cpu_baseline(a, "f64", 16, sample=1 << 12, runs=1)
    assert one["value"] > 0 and "one oracle run" in one["sample"] and "4096 keys" in one["sample"]
    assert cb["multicore"]["value"] > 0 and cb["multicore"]["cores"] >= 1
    assert cb["some_sort_alone"]["value"] > 0
    assert isinstance(cb["cpu_model"], str) and cb["cpu_model"]
