"""SqDet in the paper's own organisation (OS_DET_MERGE: split every sorted
sequence by binary search, merge every bucket's pieces) against the oracle,
which follows Algorithm 1 the same way: keys, payload order, splitters and
bucket sizes bit for bit, including p that are not powers of two (odd runs in
the merge passes) and duplicate-heavy inputs (ties across pieces)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1608_08648_gb300 as oss
from paper_1608_08648_gb300 import inputs
from tests import refcheck as rc
from tests.test_gpu_parity import gen, to_np

pytestmark = pytest.mark.gpu


def check(keys, kt, p, s, seed, with_vals=True):
    n = len(keys)
    vals = np.arange(n, dtype=np.uint32)
    o = oracle.sort(keys, kt, "det", p, s, seed=seed, vals=vals)
    src = keys.view(np.int64) if kt == "u64" else keys
    d = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    v = torch.arange(n, dtype=torch.int32, device="cuda") if with_vals else None
    ko, vo, st = oss.sort(d, v, split="det", p=p, s=s, seed=seed, key_type=kt, stats=True, det_merge=True)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(ko, kt).view(np.uint8), o["keys"].view(np.uint8)), "keys differ"
    if with_vals:
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), o["vals"]), "payload differs"
    assert st["p_used"] == o["p_used"]
    assert np.array_equal(st["bucket_sizes"], o["bucket_sizes"]), "bucket sizes differ"
    assert np.array_equal(st["spl_keys"].view(np.uint8), o["spl_keys"].view(np.uint8))
    assert np.array_equal(st["spl_tags"], o["spl_tags"])
    return st


def test_c1_det_merge_exact():
    keys = gen("uniform", 1 << 20, "i32", seed=1)
    st = check(keys, "i32", 64, 8, seed=1)
    assert st["max_bucket"] <= rc.derived_det_bound(1 << 20, 64, 8)


@pytest.mark.parametrize("kt", ["i32", "u64", "f64"])
@pytest.mark.parametrize("n", [4096, 4097, 65537, 300007, 1 << 20])
def test_sizes(kt, n):
    keys = gen("uniform", n, kt, seed=n)
    check(keys, kt, 16, 2, seed=n)
    check(keys, kt, 16, 2, seed=n, with_vals=False)


@pytest.mark.parametrize("p", [2, 3, 5, 17, 100, 1000, 1024])
def test_non_power_of_two_p(p):
    n = 1 << 21
    keys = gen("dup", n, "i32", seed=p)
    check(keys, "i32", p, 1, seed=p)


@pytest.mark.parametrize("kt", ["i32", "f64"])
@pytest.mark.parametrize("dist", list(inputs.DISTRIBUTIONS))
def test_distributions(kt, dist):
    keys = gen(dist, 500_009, kt, seed=5)
    check(keys, kt, 64, 4, seed=5)


def test_f64_edges_and_hot_u64():
    check(gen("edge", 200_003, "f64", seed=7), "f64", 32, 2, seed=7)
    check(gen("hot", 400_001, "u64", seed=8), "u64", 64, 2, seed=8)


def test_same_output_as_classify_scatter_path():
    n = 1 << 24
    keys = inputs.keys("gaussian", n, "f64", seed=9, device="cuda")
    a, _, sa = oss.sort(keys, split="det", p=1024, s=2, seed=9, key_type="f64", stats=True)
    b, _, sb = oss.sort(keys, split="det", p=1024, s=2, seed=9, key_type="f64", stats=True, det_merge=True)
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int64), b.view(torch.int64))
    assert np.array_equal(sa["bucket_sizes"], sb["bucket_sizes"])
    assert np.array_equal(sa["spl_tags"], sb["spl_tags"])


@pytest.mark.parametrize("kt", ["i32", "f64"])
def test_many_pairs_per_tile(kt):
    # n just above p^2 s with s = 1: pieces of about one element, so the first
    # merge passes put thousands of (often empty) pairs into one tile
    n = 1024 * 1024 + 3
    keys = gen("uniform", n, kt, seed=21)
    st = check(keys, kt, 1024, 1, seed=21)
    assert st["p_used"] == 1024


@pytest.mark.parametrize("kt", ["i32", "f64"])
@pytest.mark.parametrize("dist", ["uniform", "dup", "staggered"])
def test_full_size_c2_equals_default_path(kt, dist):
    # C2's size (2^27 keys, p = 1024, r = 16): the split + merge organisation gives the
    # classify/scatter path's output, splitters and bucket sizes bit for bit, and the
    # output is ordered (checked on the GPU)
    n = 1 << 27
    keys = inputs.keys(dist, n, kt, seed=1, p=1024, device="cuda")
    a, _, sa = oss.sort(keys, split="det", p=1024, s=16, seed=1, key_type=kt, stats=True)
    b, _, sb = oss.sort(keys, split="det", p=1024, s=16, seed=1, key_type=kt, stats=True, det_merge=True)
    torch.cuda.synchronize()
    view = torch.int64 if kt == "f64" else torch.int32
    assert torch.equal(a.view(view), b.view(view))
    assert np.array_equal(sa["bucket_sizes"], sb["bucket_sizes"])
    assert np.array_equal(sa["spl_tags"], sb["spl_tags"])
    assert int(sb["max_bucket"]) <= rc.derived_det_bound(n, 1024, 16)
    if kt == "i32":
        assert bool((b[1:] >= b[:-1]).all())
    del a, b, keys
    torch.cuda.empty_cache()
