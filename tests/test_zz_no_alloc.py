"""os_sort_noalloc: the sort for callers that may not allocate device memory (a
framework that owns all device memory, or a path that must not allocate after
start-up).  Its workspace is a scratch array compiled into the library, shared by
every call on a device.  Checked against os_sort (caller-provided workspace) on
two calls in a row, through the C ABI; integer keys, so the comparison is exact.

This file is collected last so that a run stopping at the first failure has run
every other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import paper_1608_08648_gb300 as oss
from paper_1608_08648_gb300 import binding as B
from paper_1608_08648_gb300 import inputs

pytestmark = pytest.mark.gpu


def _reference_sort(keys, vals, prm, kt):
    n = keys.numel()
    rc, need = B.os_workspace_size(kt, n, vals is not None, prm)
    assert rc == B.OS_OK
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.empty_like(keys)
    vout = torch.empty_like(vals) if vals is not None else None
    st = torch.cuda.current_stream().cuda_stream
    rc = B.os_sort(kt, keys.data_ptr(), out.data_ptr(), vals.data_ptr() if vals is not None else None,
                   vout.data_ptr() if vout is not None else None, n, prm, ws.data_ptr(), need, st)
    assert rc == B.OS_OK
    return out, vout


def _noalloc_sort(keys, vals, prm, kt, with_stats=False):
    n = keys.numel()
    out = torch.empty_like(keys)
    vout = torch.empty_like(vals) if vals is not None else None
    st = torch.cuda.current_stream().cuda_stream
    stats = None
    if with_stats:
        # host arrays left NULL: only the counters and the device status word
        stats = B.os_stats(0, 0, 0, 0, None, None, None)
    rc = B.os_sort_noalloc(kt, keys.data_ptr(), out.data_ptr(), vals.data_ptr() if vals is not None else None,
                           vout.data_ptr() if vout is not None else None, n, prm, st, stats)
    # with statistics the call synchronizes and returns OS_ERR_DEVICE if any
    # kernel flagged an error bit in the scratch's status word
    assert rc == B.OS_OK, B.os_strerror(rc)
    return out, vout


def test_noalloc_matches_os_sort_on_two_calls_in_a_row():
    torch.cuda.init()
    cases = [
        ("i32", "ran", 1024, 16, 1_000_003, True, 1),
        ("i32", "det", 64, 8, 1 << 20, False, 2),
    ]
    for kt_name, split, p, s, n, with_vals, seed in cases:
        kt = oss.KEY_TYPES[kt_name]
        prm = oss.params(split, p, s, seed)
        keys = inputs.keys("uniform", n, kt_name, seed=seed, p=p, device="cuda")
        vals = torch.arange(n, dtype=torch.int32, device="cuda") if with_vals else None
        ref_k, ref_v = _reference_sort(keys, vals, prm, kt)
        for rep in range(2):        # the scratch keeps the previous call's contents
            got_k, got_v = _noalloc_sort(keys, vals, prm, kt, with_stats=(rep == 1))
            torch.cuda.synchronize()
            assert torch.equal(got_k, ref_k)
            if with_vals:
                assert torch.equal(got_v, ref_v)
    # a different input right after: nothing of the previous sort leaks in
    keys2 = inputs.keys("dup", 777_777, "i32", seed=5, device="cuda")
    prm2 = oss.params("ran", 256, 8, 5)
    ref2, _ = _reference_sort(keys2, None, prm2, B.OS_I32)
    got2, _ = _noalloc_sort(keys2, None, prm2, B.OS_I32, with_stats=True)
    torch.cuda.synchronize()
    assert torch.equal(got2, ref2)
    assert torch.equal(got2, torch.sort(keys2).values)


def test_noalloc_rejects_sorts_larger_than_its_scratch():
    prm = oss.params("ran", 1024, 16, 1)
    n = 1 << 26                     # needs far more than the 64 MiB scratch
    rc, need = B.os_workspace_size(B.OS_I32, n, False, prm)
    assert rc == B.OS_OK and need > B.OS_NOALLOC_SCRATCH_BYTES
    keys = torch.empty(16, dtype=torch.int32, device="cuda")   # never touched: refused first
    rc = B.os_sort_noalloc(B.OS_I32, keys.data_ptr(), keys.data_ptr(), None, None, n, prm,
                           torch.cuda.current_stream().cuda_stream)
    assert rc == B.OS_ERR_UNSUPPORTED
