"""32-byte string keys (memcmp order) on the GPU against the oracle: the sorted
records and the payload order always; the splitters and bucket sizes whenever
the first 8 bytes order the keys as all 32 do (uniform strings and the
duplicate pool, whose 32 strings differ in their first 8 bytes).  Inputs that
tie on 8, 16 or 24 bytes exercise every refinement level."""
import numpy as np
import pytest
import torch

import oracle
import paper_1608_08648_gb300 as oss
from paper_1608_08648_gb300 import inputs

pytestmark = pytest.mark.gpu

PREFIX_ORDERED = {"uniform", "dup"}


def check(dist, n, split, p, s, seed, with_vals):
    keys = inputs.strings(dist, n, seed=seed, device="cuda")
    vals = torch.arange(n, dtype=torch.int32, device="cuda") if with_vals else None
    out, vout, st = oss.sort(keys, vals, split=split, p=p, s=s, seed=seed, key_type="s32", stats=True)
    torch.cuda.synchronize()
    kh = keys.cpu().numpy()
    ref = oracle.sort(kh, "s32", split, p, s, seed=seed,
                      vals=np.arange(n, dtype=np.uint32) if with_vals else None)
    assert np.array_equal(out.cpu().numpy().reshape(-1, 32), ref["keys"]), f"{dist} {split} n={n}: records differ"
    if with_vals:
        assert np.array_equal(vout.cpu().numpy().view(np.uint32), ref["vals"]), "payload order differs"
    assert st["p_used"] == ref["p_used"]
    assert int(st["bucket_sizes"].sum()) == n
    if dist in PREFIX_ORDERED and ref["p_used"] > 1:
        assert np.array_equal(st["spl_keys"], ref["spl_keys"]), "splitter keys differ"
        assert np.array_equal(st["spl_tags"], ref["spl_tags"]), "splitter tags differ"
        assert np.array_equal(st["bucket_sizes"], ref["bucket_sizes"]), "bucket sizes differ"


@pytest.mark.parametrize("dist", list(inputs.STR_DISTRIBUTIONS))
@pytest.mark.parametrize("split", ["ran", "det"])
@pytest.mark.parametrize("with_vals", [False, True])
def test_strings_match_oracle(dist, split, with_vals):
    check(dist, 200_003, split, 64, 8, 5, with_vals)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 4097, 33_333])
def test_string_sizes(n):
    for dist in ("uniform", "prefix24"):
        if n == 0:
            keys = torch.zeros((0, 32), dtype=torch.uint8, device="cuda")
            out, _, _ = oss.sort(keys, key_type="s32", split="ran", p=16, s=4)
            assert out.numel() == 0
            continue
        check(dist, n, "ran", 16, 4, 3, True)


def test_paper_parameters_table1_grid_point():
    # n = 1,024,000 random strings, SqRan with p = 128 and s = ceil(lg^2 n) (Section 3)
    n = 1_024_000
    s = int(np.ceil(np.log2(n) ** 2))
    check("uniform", n, "ran", 128, s, 1, False)


def test_full_size_paper_workload_properties():
    # n = 32,768,000 random strings (the largest n of Table 1), p = 256, default s:
    # the output is ordered and a stable permutation of the input (checked on the GPU).
    n = 32_768_000
    s = int(np.ceil(np.log2(n) ** 2))
    keys = inputs.strings("uniform", n, seed=2, device="cuda")
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    out, vout, st = oss.sort(keys, vals, split="ran", p=256, s=s, seed=2, key_type="s32", stats=True)
    torch.cuda.synchronize()
    # big-endian words, compared as signed after flipping the sign bit
    w = out.view(n, 4, 8).flip(2).contiguous().view(torch.int64).view(n, 4) ^ (-(1 << 63))
    a, b = w[:-1], w[1:]
    lt = torch.zeros(n - 1, dtype=torch.bool, device="cuda")
    eq = torch.ones(n - 1, dtype=torch.bool, device="cuda")
    for k in range(4):
        lt |= eq & (a[:, k] < b[:, k])
        eq &= a[:, k] == b[:, k]
    assert bool((lt | eq).all()), "records out of order"
    # a permutation: the payload is, and it carries every record to its place
    assert torch.equal(torch.sort(vout).values, vals)
    assert torch.equal(out.view(n, 32), keys.view(n, 32)[vout.long()])
    # ties (if any) keep input order
    assert bool((~eq | (vout[1:] > vout[:-1])).all())
    assert st["p_used"] == 256 and int(st["bucket_sizes"].sum()) == n


def test_in_place_and_host_buffers():
    n = 100_003
    keys = inputs.strings("prefix8", n, seed=8, device="cuda")
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    ref_k, ref_v, _ = oss.sort(keys, vals, split="ran", p=32, s=8, seed=8, key_type="s32")
    k2, v2 = keys.clone(), vals.clone()
    oss.sort(k2, v2, split="ran", p=32, s=8, seed=8, key_type="s32", out=k2, values_out=v2)
    torch.cuda.synchronize()
    assert torch.equal(k2, ref_k) and torch.equal(v2, ref_v)
    # the host-buffer entry point sorts in place inside its workspace
    prm = oss.params("ran", 32, 8, 8)
    rc, need = oss.os_workspace_size_host(oss.OS_S32, n, False, prm)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h_in = keys.cpu().pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    rc = oss.os_sort_host(oss.OS_S32, h_in.data_ptr(), h_out.data_ptr(), None, None, n, prm, ws.data_ptr(), need,
                          torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    assert torch.equal(h_out, ref_k.cpu())
