"""The configurations at their full sizes, checked on the GPU against
independent recomputations (torch's own sorts, searchsorted and bincount), never
against this library:

* C2 - n = 2^27, int32 and float64, SqDet and SqRan, p = 1024, s = 16, all seven
  distributions: the output equals torch.sort of the input; the p-1 splitters
  equal the ones recomputed from their definition (random positions from the
  counter-based generator, or the regular samples of the stably sorted
  sequences); the bucket sizes equal a count of keys against those splitters in
  the tagged order; SqDet buckets respect Lemma 1.
* C3 - n = 2^28 (uint64 key, uint32 original index), 25% hot keys, stable
  SqRan: keys equal torch.sort, payload equals the stable argsort.
"""
import numpy as np
import pytest
import torch

import paper_1608_08648_gb300 as oss
from paper_1608_08648_gb300 import inputs
from tests import refcheck as rc

pytestmark = pytest.mark.gpu

N2 = 1 << 27
P, S = 1024, 16
I64_MIN = -(1 << 63)


def ord_signed(t, kt):
    """int64 tensor whose signed order is the key order (float64: totalOrder)."""
    if kt == "i32":
        return t.to(torch.int64)
    b = t.view(torch.int64)
    if kt == "u64":
        return b ^ I64_MIN
    return torch.where(b < 0, b ^ ((1 << 63) - 1), b)


def mulhi_n(u, n):
    """floor(u * n / 2^64) for int64-held unsigned u and n < 2^31, exactly."""
    hi = (u >> 32) & 0xFFFFFFFF
    lo = u & 0xFFFFFFFF
    return (hi * n + ((lo * n) >> 32)) >> 32


def sorted_tagged(ok, tag):
    """Indices that sort (ok, tag) lexicographically (two stable passes)."""
    o1 = torch.sort(tag, stable=True).indices
    o2 = torch.sort(ok[o1], stable=True).indices
    return o1[o2]


def splitters_ref(keys, kt, split, p, s, seed):
    """(key order values, tags) of the p-1 splitters from their definition."""
    n = keys.numel()
    ok = ord_signed(keys, kt)
    dev = keys.device
    if split == "ran":
        m = p * s - 1
        u = inputs.u64(seed, 1, torch.arange(m, dtype=torch.int64, device=dev))
        pos = mulhi_n(u, n)
        tok, ttag, stride = ok[pos], pos, s
    else:
        mm = s * p
        cs = torch.tensor([(k * n) // p for k in range(p + 1)], dtype=torch.int64, device=dev)
        c = n // p
        assert n % p == 0
        chunks = ok.view(p, c)
        srt = torch.sort(chunks, dim=1, stable=True)
        j = torch.arange(1, mm + 1, dtype=torch.int64, device=dev)
        loc = (j * c + mm - 1) // mm - 1                      # local ranks of the samples
        tok = srt.values[:, loc].reshape(-1)
        ttag = (cs[:-1, None] + loc[None, :]).reshape(-1)      # position in the sorted sequences
        stride = mm
    order = sorted_tagged(tok, ttag)
    pick = torch.arange(1, p, dtype=torch.int64, device=dev) * stride - 1
    return tok[order][pick], ttag[order][pick]


def det_tags(keys, kt, p):
    n = keys.numel()
    ok = ord_signed(keys, kt).view(p, n // p)
    idx = torch.sort(ok, dim=1, stable=True).indices          # local source of each sorted slot
    base = torch.arange(p, device=keys.device, dtype=torch.int64)[:, None] * (n // p)
    tags = torch.empty(n, dtype=torch.int64, device=keys.device)
    tags[(base + idx).reshape(-1)] = (base + torch.arange(n // p, device=keys.device)[None, :]).reshape(-1)
    return tags


def bucket_sizes_ref(keys, kt, tags, sok, stag, p):
    ok = ord_signed(keys, kt)
    lo = torch.searchsorted(sok, ok, right=False)
    hi = torch.searchsorted(sok, ok, right=True)
    b = lo.clone()
    tie = torch.nonzero(hi > lo).flatten()
    if tie.numel():
        pairs = torch.stack([lo[tie], hi[tie]], 1)
        uniq, inv = torch.unique(pairs, dim=0, return_inverse=True)
        for g in range(uniq.shape[0]):
            a, z = int(uniq[g, 0]), int(uniq[g, 1])
            members = tie[inv == g]
            b[members] += torch.searchsorted(stag[a:z].contiguous(), tags[members], right=False)
    return torch.bincount(b, minlength=p)


@pytest.mark.parametrize("kt", ["i32", "f64"])
@pytest.mark.parametrize("split", ["ran", "det"])
@pytest.mark.parametrize("dist", list(inputs.DISTRIBUTIONS))
def test_c2_full_size(kt, split, dist):
    seed = 1
    keys = inputs.keys(dist, N2, kt, seed=seed, p=P, device="cuda")
    out, _, st = oss.sort(keys, split=split, p=P, s=S, seed=seed, key_type=kt, stats=True)
    torch.cuda.synchronize()
    ref = torch.sort(ord_signed(keys, kt)).values
    assert torch.equal(ord_signed(out, kt), ref), "output differs from the sorted input"
    sok, stag = splitters_ref(keys, kt, split, P, S, seed)
    got_ok = ord_signed(torch.from_numpy(np.ascontiguousarray(st["spl_keys"])).to("cuda").view(
        torch.int32 if kt == "i32" else torch.float64), kt)
    assert torch.equal(got_ok, sok), "splitter keys differ"
    assert torch.equal(torch.from_numpy(st["spl_tags"].astype(np.int64)).to("cuda"), stag), "splitter tags differ"
    tags = torch.arange(N2, dtype=torch.int64, device="cuda") if split == "ran" else det_tags(keys, kt, P)
    sizes = bucket_sizes_ref(keys, kt, tags, sok, stag, P)
    assert torch.equal(torch.from_numpy(st["bucket_sizes"].astype(np.int64)).to("cuda"), sizes)
    if split == "det":
        assert st["max_bucket"] <= rc.derived_det_bound(N2, P, S)


def test_c3_stable_u64_hot_keys_full_size():
    n = 1 << 28
    keys = inputs.hot_u64_keys(n, seed=2, device="cuda")
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    out, vout, st = oss.sort(keys, vals, split="ran", p=P, s=S, seed=2, key_type="u64", stats=True)
    torch.cuda.synchronize()
    okey = ord_signed(keys, "u64")
    ref = torch.sort(okey, stable=True)
    assert torch.equal(ord_signed(out, "u64"), ref.values)
    assert torch.equal(vout.to(torch.int64), ref.indices), "payload is not in stable order"
    assert int(st["bucket_sizes"].sum()) == n


@pytest.mark.parametrize("kt,split,dist", [("i32", "ran", "uniform"), ("f64", "ran", "gaussian"),
                                           ("i32", "det", "bucket")])
def test_c2_full_size_against_oracle_splitters(kt, split, dist):
    """The oracle itself at 2^27 keys, without its final merge: the splitters and
    the p bucket sizes it reports equal the GPU's."""
    import oracle
    seed = 3
    keys = inputs.keys(dist, N2, kt, seed=seed, p=P, device="cuda")
    _, _, st = oss.sort(keys, split=split, p=P, s=S, seed=seed, key_type=kt, stats=True)
    torch.cuda.synchronize()
    ref = oracle.sort(keys.cpu().numpy(), kt, split, P, S, seed=seed, merge=False)
    assert ref["p_used"] == st["p_used"] == P
    assert np.array_equal(ref["spl_keys"].view(np.uint8), np.ascontiguousarray(st["spl_keys"]).view(np.uint8))
    assert np.array_equal(ref["spl_tags"], st["spl_tags"])
    assert np.array_equal(ref["bucket_sizes"], st["bucket_sizes"])
