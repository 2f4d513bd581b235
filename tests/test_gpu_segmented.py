"""Batched segmented sort on the GPU (os_sort_segmented, its CUDA graph and its
autotuner), checked segment by segment against the CPU oracle: every segment's
output, payload order, splitters and bucket sizes equal what the oracle's SqRan
gives for that segment alone with the parameters of its length class and the
segment's seed."""
import numpy as np
import pytest
import torch

import oracle
import paper_1608_08648_gb300 as oss
from paper_1608_08648_gb300 import binding as B
from paper_1608_08648_gb300 import inputs
from tests import segref

pytestmark = pytest.mark.gpu

CAP = {"i32": 8192, "u64": 4096, "f64": 4096}
NP_DT = {"i32": np.int32, "u64": np.uint64, "f64": np.float64}


def mixed_lengths(kt, extra=40, seed=11):
    c = CAP[kt]
    fixed = [0, 1, 2, 17, 100, 1023, c - 1, c, c + 1, 2 * c + 5, 3 * c, 20000, 65537, 150001, 300000, 0, 5]
    u = inputs.u64(seed, 5, torch.arange(extra, dtype=torch.int64))
    rnd = [int(2 ** (17.6 * ((int(x) & ((1 << 53) - 1)) / 2 ** 53))) for x in u.tolist()]
    return fixed + rnd


TABLES = {
    "four_classes": lambda c: [(c, 1, 1, 4096), (4 * c, 2, 16, 2048), (1 << 17, 8, 32, 4096),
                               (1 << 20, 16, 64, 8192)],
    "whole_up_to_3cap": lambda c: [(3 * c, 1, 1, 4096), (1 << 20, 16, 16, 4096)],
}


def run_batch(kt, lengths, classes, seed, dist="uniform", with_vals=False):
    off = inputs.segment_offsets(torch.tensor(lengths, dtype=torch.int64))
    n = int(off[-1])
    keys = inputs.keys(dist, n, kt, seed=seed, device="cuda")
    vals = torch.arange(n, dtype=torch.int32, device="cuda") if with_vals else None
    out, vout, st = oss.sort_segmented(keys, off.cuda(), vals, classes=classes, seed=seed, key_type=kt, stats=True)
    torch.cuda.synchronize()
    return off, keys, vals, out, vout, st


def check_against_oracle(kt, classes, seed, off, keys, vals, out, vout, st, segs=None):
    kh = keys.cpu().numpy().view(NP_DT[kt])
    oh = out.cpu().numpy().view(NP_DT[kt])
    vh = vals.cpu().numpy().view(np.uint32) if vals is not None else None
    voh = vout.cpu().numpy().view(np.uint32) if vout is not None else None
    base = st["bucket_base"].cpu().numpy().astype(np.int64)
    sizes = st["bucket_sizes"].cpu().numpy().astype(np.int64)
    sk = st["splitter_keys"].cpu().numpy().view(NP_DT[kt])
    stg = st["splitter_tags"].cpu().numpy().astype(np.int64)
    nseg = off.numel() - 1
    for g in (range(nseg) if segs is None else segs):
        a, b = int(off[g]), int(off[g + 1])
        ln = b - a
        k = segref.class_of(ln, classes)
        _, pc, sc, _ = classes[k]
        ref = oracle.sort(kh[a:b], kt, "ran", pc, sc, seed=segref.seg_seed(seed, g),
                          vals=vh[a:b] if vh is not None else None)
        p_exp, _ = segref.seg_params(ln, classes)
        assert ref["p_used"] == p_exp, (g, ln)
        assert oh[a:b].tobytes() == ref["keys"].tobytes(), f"segment {g} (len {ln}): keys differ"
        if vh is not None:
            assert np.array_equal(voh[a:b], ref["vals"]), f"segment {g}: payload differs"
        b0, nb = base[g], base[g + 1] - base[g]
        assert nb == p_exp, (g, nb, p_exp)
        if p_exp == 1:
            assert sizes[b0] == ln
        else:
            assert np.array_equal(sizes[b0:b0 + nb], ref["bucket_sizes"].astype(np.int64)), f"segment {g}: sizes"
            assert sk[b0:b0 + nb - 1].tobytes() == ref["spl_keys"].tobytes(), f"segment {g}: splitter keys"
            assert np.array_equal(stg[b0:b0 + nb - 1], ref["spl_tags"].astype(np.int64)), f"segment {g}: tags"
    assert base[nseg] == sum(segref.seg_params(int(off[g + 1] - off[g]), classes)[0] for g in range(nseg))


@pytest.mark.parametrize("kt", ["i32", "u64", "f64"])
@pytest.mark.parametrize("table", list(TABLES))
@pytest.mark.parametrize("dist,with_vals", [("uniform", False), ("dup", True)])
def test_mixed_batch_matches_oracle(kt, table, dist, with_vals):
    classes = TABLES[table](CAP[kt])
    lengths = mixed_lengths(kt)
    seed = 7
    res = run_batch(kt, lengths, classes, seed, dist, with_vals)
    check_against_oracle(kt, classes, seed, *res)


def test_narrow_int32_segments():
    """int32 segments whose leaves span at most 2^16 values (the packed 16-bit
    leaf sort, also on whole segments sorted directly by the leaf kernel)."""
    kt = "i32"
    classes = TABLES["whole_up_to_3cap"](CAP[kt])
    lengths = mixed_lengths(kt, seed=13)
    off = inputs.segment_offsets(torch.tensor(lengths, dtype=torch.int64))
    n = int(off[-1])
    keys = inputs.narrow_i32_keys(n, -(1 << 15), 1 << 16, seed=5, device="cuda")
    out, _, st = oss.sort_segmented(keys, off.cuda(), classes=classes, seed=5, key_type=kt, stats=True)
    torch.cuda.synchronize()
    check_against_oracle(kt, classes, 5, off, keys, None, out, None, st)


def test_edge_f64_values_and_single_segment():
    # signed zeros, infinities and subnormals, in one segment and split in many
    n = 200_003
    keys = inputs.edge_f64_keys(n, seed=9, device="cuda")
    classes = [(4096, 1, 1, 4096), (1 << 20, 32, 16, 2048)]
    for lengths in ([n], [n // 3, n // 3, n - 2 * (n // 3)], [1] * 1000 + [n - 1000]):
        off = inputs.segment_offsets(torch.tensor(lengths))
        out, _, st = oss.sort_segmented(keys, off.cuda(), classes=classes, seed=4, key_type="f64", stats=True)
        torch.cuda.synchronize()
        check_against_oracle("f64", classes, 4, off, keys, None, out, None, st)


def _per_segment_sorted(keys, off, kt):
    """torch reference: stable sort by key inside each segment (two stable passes)."""
    n = keys.numel()
    lens = off[1:] - off[:-1]
    seg = torch.repeat_interleave(torch.arange(lens.numel(), device=keys.device), lens.to(keys.device))
    if kt == "i32":
        ok = keys.to(torch.int64)
    else:
        b = keys.view(torch.int64)
        ok = torch.where(b < 0, b ^ ((1 << 63) - 1), b) if kt == "f64" else b ^ (-(1 << 63))
    p1 = torch.sort(ok, stable=True).indices
    p2 = torch.sort(seg[p1], stable=True).indices
    assert seg.numel() == n
    return p1[p2]


def test_graph_replay_with_new_keys_and_offsets():
    kt = "f64"
    lengths = mixed_lengths(kt, extra=150, seed=12)
    off = inputs.segment_offsets(torch.tensor(lengths))
    n = int(off[-1])
    keys = inputs.keys("gaussian", n, kt, seed=3, device="cuda")
    d_off = off.cuda()
    out = torch.empty_like(keys)
    classes = oss.default_classes(kt, max(lengths))
    g = oss.SegmentedGraph(keys, d_off, out, classes=classes, seed=3)
    assert g.kernels >= 8
    before = B.os_launch_count()
    g.launch()
    torch.cuda.synchronize()
    assert B.os_launch_count() - before == g.kernels
    ref, _, _ = oss.sort_segmented(keys, d_off, classes=classes, seed=3)
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int64), ref.view(torch.int64))
    # new contents at the captured addresses: other keys, another segmentation of the same n
    keys.copy_(inputs.keys("uniform", n, kt, seed=8, device="cuda"))
    lengths2 = list(reversed(lengths))
    d_off.copy_(inputs.segment_offsets(torch.tensor(lengths2)).cuda())
    g.launch()
    torch.cuda.synchronize()
    perm = _per_segment_sorted(keys, d_off, kt)
    assert torch.equal(out.view(torch.int64), keys[perm].view(torch.int64))
    g.close()


def test_tuner_returns_a_valid_table_that_sorts():
    kt = "f64"
    L, _ = inputs.segment_lengths(300, 1024, 1 << 18, cap=1 << 23, seed=5)
    off = inputs.segment_offsets(L)
    n = int(off[-1])
    keys = inputs.keys("gaussian", n, kt, seed=5, device="cuda")
    classes, ms = oss.tune_segmented(keys, off.cuda(), seed=5, reps=1)
    assert ms > 0 and len(classes) >= 2 and classes[0][1] == 1
    assert [c[0] for c in classes] == sorted(set(c[0] for c in classes))
    for _, p, s, tile in classes[1:]:
        assert 2 <= p <= 1024 and p * s <= B.OS_SEG_MAX_PS and tile in (2048, 4096, 8192, 16384)
    out, _, st = oss.sort_segmented(keys, off.cuda(), classes=classes, seed=5, key_type=kt, stats=True)
    torch.cuda.synchronize()
    check_against_oracle(kt, classes, 5, off, keys, None, out, None, st, segs=range(0, 300, 7))
    perm = _per_segment_sorted(keys, off.cuda(), kt)
    assert torch.equal(out.view(torch.int64), keys[perm].view(torch.int64))


def test_batched_workload_full_size():
    """10,000 float64 Gaussian arrays, log-uniform lengths compressed to 2^28 keys in
    total, seed 3, the default class table."""
    kt = "f64"
    L, gamma = inputs.segment_lengths(10000, 1024, 4194304, 1 << 28, seed=3)
    off = inputs.segment_offsets(L)
    n = int(off[-1])
    keys = inputs.keys("gaussian", n, kt, seed=3, device="cuda")
    classes = oss.default_classes(kt, int(L.max()))
    out, _, st = oss.sort_segmented(keys, off.cuda(), classes=classes, seed=3, key_type=kt, stats=True)
    torch.cuda.synchronize()
    perm = _per_segment_sorted(keys, off.cuda(), kt)
    assert torch.equal(out.view(torch.int64), keys[perm].view(torch.int64))
    del perm
    big = int(torch.argmax(L))
    segs = sorted({0, 1, 9999, big, int(torch.argmin(L))} | set(range(17, 10000, 997)))
    check_against_oracle(kt, classes, 3, off, keys, None, out, None, st, segs=segs)


def test_offsets_violation_is_reported_not_faulted():
    # off[0] != 0 and off[nseg] != n: flagged in the status word; the segments that
    # are well formed are still sorted, the keys outside every segment untouched.
    n = 50_000
    keys = inputs.keys("uniform", n, "i32", seed=2, device="cuda")
    off = torch.tensor([5, 20_000, n - 3], dtype=torch.int64, device="cuda")
    classes = [(8192, 1, 1, 4096), (1 << 20, 4, 16, 2048)]
    rc, need = B.os_workspace_size_segmented(B.OS_I32, n, 2, False, classes)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.full_like(keys, 7)
    st = torch.cuda.current_stream().cuda_stream
    rc = B.os_sort_segmented(B.OS_I32, keys.data_ptr(), out.data_ptr(), None, None, n, off.data_ptr(), 2, classes, 1,
                             ws.data_ptr(), need, st)
    assert rc == B.OS_OK
    rc, bits = B.os_check(ws.data_ptr(), st)
    assert rc == B.OS_ERR_DEVICE and bits & 16
    assert torch.equal(out[5:20_000], torch.sort(keys[5:20_000]).values)
    assert torch.equal(out[20_000:n - 3], torch.sort(keys[20_000:n - 3]).values)
    assert int(out[0]) == 7 and int(out[n - 1]) == 7


def test_largest_segment_count_tiny_and_empty_segments():
    # OS_SEG_MAX_NSEG segments of 0..7 keys (about one in eight empty), int32 keys
    # with their index as payload: every segment sorted on its own, stably
    nseg = B.OS_SEG_MAX_NSEG
    u = inputs.u64(21, 9, torch.arange(nseg, dtype=torch.int64, device="cuda"))
    lengths = (u & 7).to(torch.int64)
    off = torch.zeros(nseg + 1, dtype=torch.int64, device="cuda")
    off[1:] = torch.cumsum(lengths, 0)
    n = int(off[-1])
    keys = inputs.keys("dup", n, "i32", seed=21, device="cuda")
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    out, vout, _ = oss.sort_segmented(keys, off, vals, seed=21)
    torch.cuda.synchronize()
    perm = _per_segment_sorted(keys, off, "i32")
    assert torch.equal(out, keys[perm]), "keys differ from the per-segment stable sort"
    assert torch.equal(vout, vals[perm]), "payload order differs (stability)"
    del keys, vals, out, vout, perm
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kt", ["i32", "u64", "f64"])
@pytest.mark.parametrize("dist,with_vals", [("dup", True), ("uniform", False)])
def test_small_leaves_at_warp_sort_boundaries(kt, dist, with_vals):
    # whole segments of at most 256 keys are sorted by one warp each (bitonic
    # networks of 32, 64, 128 or 256); lengths around every boundary, and above
    # 256 (a CTA), each several times
    base = [1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 300, 0,
            511, 512, 513, 1023, 1024, 1025, 2000]
    lengths = base * 7
    off = inputs.segment_offsets(torch.tensor(lengths)).cuda()
    n = int(off[-1])
    keys = inputs.keys(dist, n, kt, seed=17, device="cuda")
    vals = torch.arange(n, dtype=torch.int32, device="cuda") if with_vals else None
    out, vout, _ = oss.sort_segmented(keys, off, vals, seed=17, key_type=kt)
    torch.cuda.synchronize()
    perm = _per_segment_sorted(keys, off, kt)
    view = torch.int32 if kt == "i32" else torch.int64
    assert torch.equal(out.view(view), keys[perm].view(view))
    if with_vals:
        assert torch.equal(vout, vals[perm])
