"""Sorting host buffers (os_sort_host): the keys are copied in, sorted, and the
output is copied back -- for large inputs range by range while later bucket
ranges are still being sorted.  The result must equal the device sort's, keys
and payload, for every key type and splitter choice, above and below the size
where the ranges start (2^22 keys), and for an input too small to sample."""
import pytest
import torch

import paper_1608_08648_gb300 as oss
from paper_1608_08648_gb300 import inputs

pytestmark = pytest.mark.gpu


def host_sort(keys_cpu, vals_cpu, kt, split, p, s, seed):
    n = keys_cpu.numel()
    prm = oss.params(split, p, s, seed)
    rc, need = oss.os_workspace_size_host(oss.KEY_TYPES[kt], n, vals_cpu is not None, prm)
    assert rc == 0
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")
    h_in = keys_cpu.pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    h_vin = vals_cpu.pin_memory() if vals_cpu is not None else None
    h_vout = torch.empty_like(h_vin).pin_memory() if vals_cpu is not None else None
    rc = oss.os_sort_host(oss.KEY_TYPES[kt], h_in.data_ptr(), h_out.data_ptr(),
                          h_vin.data_ptr() if h_vin is not None else None,
                          h_vout.data_ptr() if h_vout is not None else None, n, prm, ws.data_ptr(), need,
                          torch.cuda.current_stream().cuda_stream)
    assert rc == 0, rc
    return h_out, h_vout


@pytest.mark.parametrize("kt", ["i32", "u64", "f64"])
@pytest.mark.parametrize("split", ["ran", "det"])
@pytest.mark.parametrize("n", [(1 << 22) + 12345, 300_007, 100])
def test_host_buffers_equal_device_sort(kt, split, n):
    dist = "dup" if kt == "i32" else "uniform"
    keys = inputs.keys(dist, n, kt, seed=n % 97, device="cuda")
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    p, s = (256, 8) if split == "ran" else (64, 4)
    for with_vals in (False, True):
        d_out, d_vout, _ = oss.sort(keys, vals if with_vals else None, split=split, p=p, s=s, seed=3, key_type=kt)
        torch.cuda.synchronize()
        h_out, h_vout = host_sort(keys.cpu(), vals.cpu() if with_vals else None, kt, split, p, s, 3)
        view = torch.int32 if kt == "i32" else torch.int64
        assert torch.equal(h_out.view(view), d_out.cpu().view(view)), f"{kt} {split} n={n}: keys differ"
        if with_vals:
            assert torch.equal(h_vout, d_vout.cpu()), f"{kt} {split} n={n}: payload differs"


@pytest.mark.parametrize("kt", ["i32", "f64"])
def test_host_buffers_in_place_and_pageable(kt):
    # page-locked input sorted in place (the sort reads it directly and writes the
    # result back into it), and a pageable input (copied in first)
    n = (1 << 22) + 7
    keys = inputs.keys("uniform", n, kt, seed=21, device="cuda")
    d_out, _, _ = oss.sort(keys, split="ran", p=512, s=16, seed=4, key_type=kt)
    torch.cuda.synchronize()
    view = torch.int32 if kt == "i32" else torch.int64
    prm = oss.params("ran", 512, 16, 4)
    rc, need = oss.os_workspace_size_host(oss.KEY_TYPES[kt], n, False, prm)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    h = keys.cpu().pin_memory()
    assert oss.os_sort_host(oss.KEY_TYPES[kt], h.data_ptr(), h.data_ptr(), None, None, n, prm, ws.data_ptr(), need,
                            st) == 0
    assert torch.equal(h.view(view), d_out.cpu().view(view))
    pg = keys.cpu()
    assert not pg.is_pinned()
    out = torch.empty_like(pg)
    assert oss.os_sort_host(oss.KEY_TYPES[kt], pg.data_ptr(), out.data_ptr(), None, None, n, prm, ws.data_ptr(), need,
                            st) == 0
    assert torch.equal(out.view(view), d_out.cpu().view(view))
