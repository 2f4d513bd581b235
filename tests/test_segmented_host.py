"""Host-side parts of the batched segmented sort: the length generator of the
batched workload, the default class table, workspace planning and argument
checks (no GPU)."""
import math

import pytest
import torch

from paper_1608_08648_gb300 import binding as B
from paper_1608_08648_gb300 import build as _build
from paper_1608_08648_gb300 import inputs
from tests import segref


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return B.lib()


def test_segment_lengths_of_the_batched_workload():
    # 10,000 arrays log-uniform in [2^10, 2^22] capped at 2^28 keys in total.
    L, gamma = inputs.segment_lengths(10000, 1024, 4194304, 1 << 28, seed=3)
    assert L.numel() == 10000
    assert int(L.sum()) <= 1 << 28
    assert int(L.min()) >= 1024
    assert 0.55 < gamma < 0.62                      # the uncapped total is about 5e9
    assert 100_000 < int(L.max()) < 160_000
    # gamma is the largest that fits: a slightly larger one overflows the cap
    Lraw, g1 = inputs.segment_lengths(10000, 1024, 4194304, 1 << 62, seed=3)
    assert g1 == 1.0
    bigger = torch.floor(1024 * torch.pow(Lraw.to(torch.float64) / 1024, gamma + 1e-6)).to(torch.int64)
    assert int(bigger.sum()) > 1 << 28
    # uncapped lengths are log-uniform: about half of them fall below the geometric mid-point
    frac = float((Lraw < math.sqrt(1024 * 4194304)).double().mean())
    assert 0.47 < frac < 0.53
    assert int(Lraw.min()) >= 1024 and int(Lraw.max()) < 4194304


def test_segment_offsets():
    off = inputs.segment_offsets(torch.tensor([3, 0, 5]))
    assert off.tolist() == [0, 3, 3, 8]


@pytest.mark.parametrize("kt,cap", [(B.OS_I32, 8192), (B.OS_F64, 4096), (B.OS_U64, 4096)])
def test_default_classes(lib, kt, cap):
    for max_len in (10, cap, cap + 1, 132053, 1 << 22, (1 << 31) - 1):
        rc, cl = B.os_seg_default_classes(kt, max_len)
        assert rc == B.OS_OK
        assert cl[0].max_len == cap and cl[0].p == 1
        lens = [c.max_len for c in cl]
        assert lens == sorted(set(lens))
        assert cl[-1].max_len == max(cap, max_len)
        for k in range(1, len(cl)):
            c, lo = cl[k], cl[k - 1].max_len
            assert c.p >= 2 and (c.p & (c.p - 1)) == 0 and c.p <= 256
            assert 2 * c.p * c.s <= lo + 1 or c.p == 2   # the shortest segment of the class is sampled
            assert c.p * c.s <= B.OS_SEG_MAX_PS and c.tile % 2048 == 0
    rc, cl = B.os_seg_default_classes(kt, 1 << 22, max_classes=3)
    assert rc == B.OS_OK and len(cl) == 3 and cl[-1].max_len == 1 << 22


def test_workspace_and_argument_checks(lib):
    good = [(4096, 1, 1, 4096), (1 << 20, 16, 16, 2048)]
    rc, b = B.os_workspace_size_segmented(B.OS_F64, 1 << 20, 100, False, good)
    assert rc == B.OS_OK and b > 8 << 20
    rc2, b2 = B.os_workspace_size_segmented(B.OS_F64, 1 << 20, 100, True, good)
    assert rc2 == B.OS_OK and b2 > b
    rc3, b3 = B.os_workspace_size_segmented(B.OS_F64, 1 << 20, 100, False, None)
    assert rc3 == B.OS_OK and b3 >= b
    bad_tables = [
        [(4096, 1, 1, 1000)],                      # tile not a multiple of 2048
        [(4096, 1, 1, 32768)],                     # tile too large
        [(4096, 128, 64, 4096)],                   # p s above the sample capacity
        [(4096, 0, 1, 4096)],                      # p = 0
        [(4096, 2, 0, 4096)],                      # s = 0
        [(8192, 2, 4, 4096), (4096, 2, 4, 4096)],  # max_len not increasing
        [(8192, 8192, 1, 4096)],                   # p above OS_MAX_P
        [],
    ]
    for t in bad_tables:
        assert B.os_workspace_size_segmented(B.OS_F64, 1000, 3, False, t)[0] == B.OS_ERR_ARG, t
    assert B.os_workspace_size_segmented(9, 1000, 3, False, good)[0] == B.OS_ERR_ARG
    assert B.os_workspace_size_segmented(B.OS_F64, (1 << 31) + 1, 3, False, good)[0] == B.OS_ERR_UNSUPPORTED
    assert B.os_workspace_size_segmented(B.OS_F64, 1000, (1 << 26) + 1, False, good)[0] == B.OS_ERR_UNSUPPORTED
    # refused before any device work: overlapping in/out, missing offsets, n without segments
    assert B.os_sort_segmented(B.OS_F64, 4096, 4096, None, None, 100, 8192, 1, good, 0, 1 << 20, 1 << 30,
                               None) == B.OS_ERR_ARG
    assert B.os_sort_segmented(B.OS_F64, 4096, 8192, None, None, 100, None, 1, good, 0, 1 << 20, 1 << 30,
                               None) == B.OS_ERR_ARG
    assert B.os_sort_segmented(B.OS_F64, 4096, 8192, None, None, 100, 8192, 0, good, 0, 1 << 20, 1 << 30,
                               None) == B.OS_ERR_ARG
    assert B.os_sort_segmented(B.OS_F64, 4096, 8192, 16384, None, 100, 8192, 1, good, 0, 1 << 20, 1 << 30,
                               None) == B.OS_ERR_ARG
    # workspace too small
    assert B.os_sort_segmented(B.OS_F64, 4096, 8192, None, None, 100, 8192, 1, good, 0, 1 << 20, 16,
                               None) == B.OS_ERR_WS
    # graph capture and tuner check their arguments first too
    assert B.os_graph_capture_segmented(B.OS_F64, 4096, 4096, None, None, 100, 8192, 1, good, 0, 1 << 20,
                                        1 << 30)[0] == B.OS_ERR_ARG
    assert B.os_graph_launch(None, None) == B.OS_ERR_ARG
    assert B.os_graph_destroy(None) == B.OS_ERR_ARG


def test_segment_rule_of_the_tests():
    classes = [(4096, 1, 1, 4096), (8192, 2, 16, 4096), (1 << 20, 8, 64, 2048)]
    assert segref.seg_params(0, classes) == (1, 1)
    assert segref.seg_params(4096, classes) == (1, 1)
    assert segref.seg_params(4097, classes) == (2, 16)
    assert segref.seg_params(8193, classes) == (8, 64)
    assert segref.seg_params(1023, [(10, 4, 128, 2048), (2000, 4, 128, 2048)]) == (1, 128)   # 1023 < 2 p s
    assert segref.seg_params(1 << 22, classes) == (8, 64)                                 # beyond the last class
    assert segref.seg_seed(3, 0) == inputs.u64(3, 2, torch.tensor([0])).item() & ((1 << 64) - 1)
