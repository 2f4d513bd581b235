"""Pins of the CPU oracle against facts outside itself (no GPU needed).

Each test pins a part of the oracle to something it does not compute itself:
the published SplitMix64 outputs, the IEEE 754 totalOrder bit map, numpy's
stable sorts (brute force), hand-worked SqDet examples (tests/golden), the
Lemma 1 bucket bound, the regular-sampling bound of the r = 1 case and the
Claim 1 balance bound of SqRan.
"""
import glob
import itertools
import math
import os
import struct

import numpy as np
import pytest
import torch

import oracle
from paper_1608_08648_gb300 import inputs
from tests import refcheck as rc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---- random numbers ----------------------------------------------------------

def test_splitmix64_published_outputs():
    # First five outputs of the SplitMix64 reference generator started from state 0
    # (Steele, Lea and Flood, OOPSLA 2014; the widely reproduced splitmix64.c).
    published = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                 0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [oracle.splitmix64_raw(0, i) for i in range(5)] == published


def test_splitmix64_streams_agree_with_generator_module():
    idx = torch.tensor([0, 1, 2, 1000, 123456789, (1 << 40) + 7], dtype=torch.int64)
    for seed in (0, 1, 2, 3, 0xDEADBEEF):
        for stream in (0, 1, 11, 74):
            ref = inputs.u64(seed, stream, idx).numpy().view(np.uint64)
            got = [oracle.splitmix64(seed, stream, int(i)) for i in idx]
            assert got == [int(x) for x in ref]


def test_ran_index_range_and_uniformity():
    n = 1000
    seen = np.array([oracle.ran_index(5, j, n) for j in range(20000)])
    assert seen.min() >= 0 and seen.max() < n
    counts = np.bincount(seen // 100, minlength=10)
    chi2 = float(((counts - 2000.0) ** 2 / 2000.0).sum())
    assert chi2 < 30.0                     # 9 dof: p ~ 4e-4
    for j in (0, 1, 77):
        u = oracle.splitmix64(5, 1, j)
        assert oracle.ran_index(5, j, 1 << 32) == u >> 32


# ---- key order ---------------------------------------------------------------

def _f64_bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def test_f64_total_order_special_values():
    vals = [-math.inf, -1.7976931348623157e308, -1.0, -2.2250738585072014e-308,
            -2.225073858507201e-308, -5e-324, -0.0, 0.0, 5e-324, 2.225073858507201e-308,
            2.2250738585072014e-308, 1.0, 1.7976931348623157e308, math.inf]
    bits = [_f64_bits(v) for v in vals]
    for a, b in itertools.combinations(range(len(vals)), 2):
        assert oracle.key_cmp("f64", bits[a], bits[b]) == -1
        assert oracle.key_cmp("f64", bits[b], bits[a]) == 1
    for b in bits:
        assert oracle.key_cmp("f64", b, b) == 0


def test_key_order_matches_bit_maps():
    keys = {
        "i32": inputs.keys("uniform", 3000, "i32", seed=4).numpy() - (1 << 30),
        "u64": inputs.keys("uniform", 3000, "u64", seed=4).numpy().view(np.uint64),
        "f64": inputs.edge_f64_keys(3000, seed=4).numpy(),
    }
    for kt, k in keys.items():
        k = k.astype(rc.NP_DT[kt])
        ok = rc.order_key(k, kt)
        raw = k.view(np.uint32).astype(np.uint64) if kt == "i32" else k.view(np.uint64)
        for a, b in zip(range(0, 3000, 2), range(1, 3000, 2)):
            want = int(ok[a] > ok[b]) - int(ok[a] < ok[b])
            assert oracle.key_cmp(kt, int(raw[a]), int(raw[b])) == want


# ---- output and intermediates vs brute force ---------------------------------

def _check_run(keys, kt, split, p, s, seed, check_bound=True):
    n = len(keys)
    vals = np.arange(n, dtype=np.uint32)
    r = oracle.sort(keys, kt, split, p, s, seed=seed, vals=vals)
    perm = rc.brute_perm(keys, kt)
    assert np.array_equal(r["vals"], perm.astype(np.uint32))
    assert np.array_equal(r["keys"].view(np.uint8), keys[perm].view(np.uint8))
    sizes = r["bucket_sizes"]
    assert int(sizes.sum()) == n
    if r["p_used"] == 1:
        return r
    el, tg = rc.splitters(keys, kt, split, p, s, seed)
    assert np.array_equal(r["spl_keys"].view(np.uint8), keys[el].view(np.uint8))
    assert np.array_equal(r["spl_tags"], tg.astype(np.uint64))
    tags = rc.det_tags(keys, kt, p) if split == "det" else np.arange(n)
    b = rc.bucket_of(keys, kt, tags, el, tg)
    assert np.array_equal(np.bincount(b, minlength=p), sizes.astype(np.int64))
    if split == "det" and check_bound:
        assert int(sizes.max()) <= rc.derived_det_bound(n, p, s)
    return r


def test_exhaustive_small_inputs():
    """Every int32 input of length 3..7 over the alphabet {0, 1, 2}."""
    for n in range(3, 8):
        for t in itertools.product((0, 1, 2), repeat=n):
            keys = np.array(t, dtype=np.int32)
            _check_run(keys, "i32", "det", 2, 1, 0)
            if n >= 4:
                _check_run(keys, "i32", "ran", 2, 1, n)


@pytest.mark.parametrize("kt", ["i32", "u64", "f64"])
@pytest.mark.parametrize("split", ["det", "ran"])
def test_distributions_vs_brute_force(kt, split):
    for di, dist in enumerate(inputs.DISTRIBUTIONS):
        for n, p, s in ((3000, 4, 3), (20011, 16, 4), (4096, 8, 8)):
            keys = inputs.keys(dist, n, kt, seed=1 + di, p=p).numpy()
            if kt == "u64":
                keys = keys.view(np.uint64)
            _check_run(keys.astype(rc.NP_DT[kt]), kt, split, p, s, seed=di)


def test_f64_edge_values_vs_brute_force():
    keys = inputs.edge_f64_keys(6000, seed=3).numpy()
    for split in ("det", "ran"):
        _check_run(keys, "f64", split, 8, 4, seed=2)


def test_hot_u64_keys_stability():
    keys = inputs.hot_u64_keys(30000, seed=2).numpy().view(np.uint64)
    for split in ("det", "ran"):
        _check_run(keys, "u64", split, 16, 4, seed=9)


# ---- hand-worked examples -------------------------------------------------------

def _parse_golden(path):
    d = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        d[k] = v
    return d


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.txt"))),
                         ids=os.path.basename)
def test_golden_worked_examples(path):
    g = _parse_golden(path)
    kt, split = g["kt"][0], g["split"][0]
    p, s, seed = int(g["p"][0]), int(g["s"][0]), int(g["seed"][0])
    keys = np.array([int(x) for x in g["keys"]], dtype=rc.NP_DT[kt])
    r = oracle.sort(keys, kt, split, p, s, seed=seed)
    assert [int(x) for x in r["spl_keys"]] == [int(x) for x in g["splitter_keys"]]
    assert [int(x) for x in r["spl_tags"]] == [int(x) for x in g["splitter_tags"]]
    assert [int(x) for x in r["bucket_sizes"]] == [int(x) for x in g["bucket_sizes"]]
    assert np.array_equal(r["keys"], np.sort(keys))


# ---- bounds from the paper -------------------------------------------------------

def test_lemma1_closed_form_when_padding_is_exact():
    """Lemma 1: n_max <= (1 + 1/r) n/p + r p, here with p | n and r p | n/p."""
    p, r = 16, 4
    n = p * (r * p) * 32
    bound = (1 + 1 / r) * n / p + r * p
    for dist in inputs.DISTRIBUTIONS:
        keys = inputs.keys(dist, n, "i32", seed=5, p=p).numpy()
        sizes = oracle.sort(keys, "i32", "det", p, r, merge=False)["bucket_sizes"]
        assert sizes.max() <= bound
        assert sizes.max() <= rc.derived_det_bound(n, p, r)


def test_regular_sampling_case_r1():
    """r = 1 is regular sampling (p samples per sequence): every bucket is at most
    about 2n/p (Lemma 1 at r = 1: 2 n/p + p)."""
    for seed in range(6):
        for dist in ("uniform", "zero", "bucket", "staggered", "dup"):
            n, p = 40000 + seed, 32
            keys = inputs.keys(dist, n, "i32", seed=seed, p=p).numpy()
            sizes = oracle.sort(keys, "i32", "det", p, 1, merge=False)["bucket_sizes"]
            assert sizes.max() <= 2 * (n / p) + p


def test_claim1_balance_at_default_oversampling():
    """Claim 1 with rho = 1 at s = ceil(lg^2 n): no bucket above ceil((1+eps)(n-p+1)/p)."""
    n, p = 1 << 16, 16
    s = math.ceil(math.log2(n) ** 2)
    rho = 1.0
    L = 2 * rho * math.log(n) + math.log(2 * math.pi * p * p * (p * s - 1)
                                         * math.exp(1 / (3 * (p * s - 1))))
    eps = (1 + math.sqrt(1 + 4 * s / L)) / (2 * s / L)      # smallest eps with s = (1+eps)L/eps^2
    limit = math.ceil((1 + eps) * (n - p + 1) / p)
    for seed in range(12):
        keys = inputs.keys("uniform", n, "i32", seed=seed).numpy()
        sizes = oracle.sort(keys, "i32", "ran", p, s, seed=seed, merge=False)["bucket_sizes"]
        assert sizes.max() <= limit


def test_too_small_inputs_form_one_bucket():
    keys = inputs.keys("uniform", 100, "i32", seed=1).numpy()
    r = oracle.sort(keys, "i32", "ran", 8, 8)           # n < 2 p s
    assert r["p_used"] == 1 and int(r["bucket_sizes"][0]) == 100
    r = oracle.sort(keys, "i32", "det", 8, 2)           # ceil(n/p) = 13 < r p = 16
    assert r["p_used"] == 1
    assert np.array_equal(r["keys"], np.sort(keys))
    r = oracle.sort(keys[:0], "i32", "det", 8, 2)
    assert r["keys"].shape == (0,)
