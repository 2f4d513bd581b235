"""The largest inputs the ABI accepts (n = OS_MAX_N = 2^31 int32 keys), checked on
the GPU by properties that hold at any size: the output is ordered, it holds the
same keys (histograms of the high and low 16 bits and the sum agree), the bucket
sizes add up to n; with a payload (2^30 keys, original index), equal keys keep
their input order and the payload carries every key to its place."""
import pytest
import torch

import paper_1608_08648_gb300 as oss
from paper_1608_08648_gb300 import binding as B
from paper_1608_08648_gb300 import inputs

pytestmark = pytest.mark.gpu


def same_keys(a, b):
    for shift in (16, 0):
        ha = torch.bincount(((a.to(torch.int64) >> shift) & 0xFFFF), minlength=65536)
        hb = torch.bincount(((b.to(torch.int64) >> shift) & 0xFFFF), minlength=65536)
        if not torch.equal(ha, hb):
            return False
    return int(a.to(torch.int64).sum()) == int(b.to(torch.int64).sum())


@pytest.mark.parametrize("split", ["ran", "det"])
def test_largest_n_int32(split):
    n = B.OS_MAX_N
    keys = inputs.keys("uniform", n, "i32", seed=13, device="cuda")
    out, _, st = oss.sort(keys, split=split, p=1024, s=16, seed=13, key_type="i32", stats=True)
    torch.cuda.synchronize()
    assert bool((out[1:] >= out[:-1]).all()), "not ordered"
    assert same_keys(keys, out), "not a permutation of the input"
    assert st["p_used"] == 1024 and int(st["bucket_sizes"].sum()) == n
    del keys, out
    torch.cuda.empty_cache()


def test_large_stable_payload():
    n = 1 << 30
    keys = inputs.keys("dup", n, "i32", seed=14, device="cuda")        # 32 distinct values: long runs of ties
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    out, vout, st = oss.sort(keys, vals, split="ran", p=1024, s=16, seed=14, key_type="i32", stats=True)
    torch.cuda.synchronize()
    assert bool((out[1:] >= out[:-1]).all())
    assert torch.equal(keys[vout.long()], out), "payload does not carry each key to its place"
    eq = out[1:] == out[:-1]
    assert bool((~eq | (vout[1:] > vout[:-1])).all()), "equal keys out of input order"
    assert torch.equal(torch.sort(vout).values, vals)
    assert int(st["bucket_sizes"].sum()) == n
