"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Every case compares, bit for bit: the sorted keys, the payload (original index,
so the payload order checks stability), the p-1 tagged splitters and the p
bucket sizes.  Sizes span several tiles of every kernel and a ragged tail.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1608_08648_gb300 as oss
from paper_1608_08648_gb300 import inputs
from tests import refcheck as rc

pytestmark = pytest.mark.gpu

TORCH_DT = {"i32": torch.int32, "u64": torch.int64, "f64": torch.float64}


def to_np(t, kt):
    a = t.cpu().numpy()
    return a.view(np.uint64) if kt == "u64" else a


def gen(dist, n, kt, seed, p=1024):
    if kt == "u64" and dist == "hot":
        return inputs.hot_u64_keys(n, seed=seed).numpy().view(np.uint64)
    if kt == "f64" and dist == "edge":
        return inputs.edge_f64_keys(n, seed=seed).numpy()
    a = inputs.keys(dist, n, kt, seed=seed, p=p).numpy()
    return a.view(np.uint64) if kt == "u64" else a


def gpu_sort(keys, kt, split, p, s, seed, with_vals=True, inplace=False):
    n = len(keys)
    src = keys.view(np.int64) if kt == "u64" else keys
    d = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    v = torch.arange(n, dtype=torch.int32, device="cuda") if with_vals else None
    out = d if inplace else None
    vout = v if (inplace and with_vals) else None
    ko, vo, st = oss.sort(d, v, split=split, p=p, s=s, seed=seed, out=out, values_out=vout,
                          key_type=kt, stats=True)
    torch.cuda.synchronize()
    return to_np(ko, kt), (vo.cpu().numpy().view(np.uint32) if with_vals else None), st


def check(keys, kt, split, p, s, seed, with_vals=True, inplace=False):
    n = len(keys)
    vals = np.arange(n, dtype=np.uint32)
    o = oracle.sort(keys, kt, split, p, s, seed=seed, vals=vals)
    gk, gv, st = gpu_sort(keys, kt, split, p, s, seed, with_vals=with_vals, inplace=inplace)
    assert np.array_equal(gk.view(np.uint8), o["keys"].view(np.uint8)), "keys differ"
    if with_vals:
        assert np.array_equal(gv, o["vals"]), "payload differs"
    assert st["p_used"] == o["p_used"]
    assert np.array_equal(st["bucket_sizes"], o["bucket_sizes"]), "bucket sizes differ"
    assert np.array_equal(st["spl_keys"].view(np.uint8), o["spl_keys"].view(np.uint8)), "splitter keys differ"
    assert np.array_equal(st["spl_tags"], o["spl_tags"]), "splitter tags differ"
    if o["p_used"] > 1:
        assert st["max_bucket"] == int(o["bucket_sizes"].max())
    return st


def test_c1_det_int32_uniform_exact():
    """n = 2^20 int32 uniform in [0, 2^31) from seed 1, SqDet p = 64, r = 8."""
    keys = gen("uniform", 1 << 20, "i32", seed=1)
    st = check(keys, "i32", "det", 64, 8, seed=1)
    assert st["max_bucket"] <= rc.derived_det_bound(1 << 20, 64, 8)


@pytest.mark.parametrize("kt", ["i32", "u64", "f64"])
@pytest.mark.parametrize("split", ["det", "ran"])
@pytest.mark.parametrize("n", [1, 2, 3, 100, 4095, 4096, 4097, 8191, 8192, 8193, 65537, 300007])
def test_sizes_across_tiles(kt, split, n):
    keys = gen("uniform", n, kt, seed=n)
    check(keys, kt, split, 4, 2, seed=n)
    check(keys, kt, split, 4, 2, seed=n, with_vals=False)
    if n >= 4097:
        check(keys, kt, split, 16, 3, seed=n + 1)
        check(keys, kt, split, 16, 3, seed=n + 1, with_vals=False)


@pytest.mark.parametrize("kt", ["i32", "u64", "f64"])
@pytest.mark.parametrize("split", ["det", "ran"])
@pytest.mark.parametrize("dist", list(inputs.DISTRIBUTIONS))
def test_distributions(kt, split, dist):
    n = (1 << 18) + 1234
    keys = gen(dist, n, kt, seed=3, p=64)
    check(keys, kt, split, 64, 8, seed=5)
    check(keys, kt, split, 64, 8, seed=5, with_vals=False)


@pytest.mark.parametrize("split", ["det", "ran"])
def test_f64_special_values(split):
    keys = gen("edge", 200003, "f64", seed=11)
    check(keys, "f64", split, 32, 4, seed=7)
    check(keys, "f64", split, 32, 4, seed=7, with_vals=False)


@pytest.mark.parametrize("split", ["det", "ran"])
def test_u64_hot_keys_stable(split):
    keys = gen("hot", (1 << 20) + 17, "u64", seed=2)
    check(keys, "u64", split, 256, 4, seed=2)


@pytest.mark.parametrize("kt", ["i32", "f64"])
def test_buckets_larger_than_a_cta(kt):
    """Few buckets: every bucket is repartitioned inside the bucket phase."""
    keys = gen("uniform", (1 << 21) + 5, kt, seed=9)
    for with_vals in (True, False):
        st = check(keys, kt, "ran", 4, 16, seed=9, with_vals=with_vals)
        assert st["depth"] >= 1
        st = check(keys, kt, "det", 8, 2, seed=9, with_vals=with_vals)
        assert st["depth"] >= 1


def test_max_p_and_non_power_of_two_p():
    keys = gen("uniform", 1 << 19, "i32", seed=4)
    check(keys, "i32", "ran", 4096, 2, seed=4)
    check(keys, "i32", "ran", 1000, 3, seed=4)
    check(keys, "i32", "det", 7, 5, seed=4)
    check(gen("uniform", 1 << 24, "i32", seed=4), "i32", "det", 4096, 1, seed=4, with_vals=False)


@pytest.mark.parametrize("split", ["det", "ran"])
def test_all_equal_keys_balance(split):
    n = (1 << 20) + 3
    keys = np.full(n, 42, dtype=np.int32)
    st = check(keys, "i32", split, 64, 8, seed=1)
    assert st["max_bucket"] <= 2 * n // 64 + 64
    check(keys, "i32", split, 64, 8, seed=1, with_vals=False)


@pytest.mark.parametrize("kt", ["i32", "f64"])
def test_in_place(kt):
    keys = gen("gaussian", (1 << 20) + 99, kt, seed=6)
    check(keys, kt, "ran", 128, 8, seed=6, inplace=True)
    check(keys, kt, "det", 32, 4, seed=6, inplace=True)


def test_keys_only():
    keys = gen("dup", (1 << 20) + 1, "i32", seed=8)
    check(keys, "i32", "ran", 256, 8, seed=8, with_vals=False)
    check(keys, "i32", "det", 64, 8, seed=8, with_vals=False)


def test_too_small_to_sample_and_p1():
    for n in (0, 1, 50, 1000, 20000):
        keys = gen("uniform", n, "i32", seed=n)
        check(keys, "i32", "ran", 64, 16, seed=1)     # n < 2 p s
        check(keys, "i32", "det", 64, 8, seed=1)      # ceil(n/p) < r p
        check(keys, "i32", "det", 1, 8, seed=1)       # p = 1


def test_status_word_clean_after_sorts():
    keys = torch.from_numpy(gen("uniform", 1 << 20, "i32", seed=1)).cuda()
    ws = torch.empty(oss.workspace_bytes(1 << 20, "i32", False, "ran", 1024, 16), dtype=torch.uint8, device="cuda")
    out, _, _ = oss.sort(keys, split="ran", p=1024, s=16, seed=3, workspace=ws)
    rc_, bits = oss.os_check(ws.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc_ == oss.OS_OK and bits == 0
    assert torch.equal(out, torch.sort(keys).values)


@pytest.mark.parametrize("kt", ["i32", "f64"])
@pytest.mark.parametrize("shift", [1, 3])
def test_keys_not_16_byte_aligned(kt, shift):
    """Input and output arrays that start off a 16-byte boundary (views into larger
    tensors): the vector passes fall back to loads of one key; the result is the
    oracle's for the same keys."""
    n = (1 << 20) + 17
    keys = gen("uniform", n, kt, seed=11 + shift)
    big = torch.from_numpy(np.concatenate([np.zeros(shift, keys.dtype), keys, np.zeros(5, keys.dtype)])).cuda()
    d = big[shift:shift + n]
    outbig = torch.empty_like(big)
    out = outbig[shift:shift + n]
    assert d.data_ptr() % 16 != 0 and out.data_ptr() % 16 != 0
    for split, p, s in (("ran", 64, 8), ("det", 32, 4)):
        ref = oracle.sort(keys, kt, split, p, s, seed=5)
        ko, _, st = oss.sort(d, None, split=split, p=p, s=s, seed=5, out=out, key_type=kt, stats=True)
        torch.cuda.synchronize()
        assert np.array_equal(to_np(ko, kt).view(np.uint8), ref["keys"].view(np.uint8)), f"{split}: keys differ"
        assert np.array_equal(st["bucket_sizes"], ref["bucket_sizes"])
        assert np.array_equal(st["spl_tags"], ref["spl_tags"])


@pytest.mark.parametrize("lo,width", [(0, 1 << 16), (-(1 << 31), 1 << 12), ((1 << 31) - (1 << 17), 1 << 17),
                                      (12345, 1 << 22), (-(1 << 20), 1 << 21)])
def test_narrow_range_leaves(lo, width):
    """Keys from a narrow range: leaves whose keys span at most 2^16 values sort
    16-bit offsets two to a register, wider ones the 32-bit elements; the cases
    mix both, put keys next to either end of the int32 range (offsets from a
    minimum close to the top stay on the 32-bit path) and include many equal
    keys."""
    for n, p, s in (((1 << 20) + 333, 64, 8), (300007, 16, 3), (8193, 4, 2), (4097, 4, 2), (100, 4, 2)):
        keys = inputs.narrow_i32_keys(n, lo, width, seed=n).numpy()
        check(keys, "i32", "ran", p, s, seed=n, with_vals=False)
        check(keys, "i32", "det", p, s, seed=n, with_vals=False)
        check(keys, "i32", "ran", p, s, seed=n)
