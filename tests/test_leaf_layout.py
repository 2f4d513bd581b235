"""Host-side checks of the leaf sort's index arithmetic (csrc/mergesort.cuh and
leaf_sort in csrc/kernels.cuh), written out in Python on small cases:

* the merge round over a bitonic pair: the second run of every pair stored
  descending, each thread's start found by a merge-path search on that layout,
  then IT outputs taken from the smaller end of the part not yet output; every
  read stays inside the pair and the outputs are the sorted union, ties included;
* the descending store: thread bases in the second run of a pair write exactly
  the mirror positions of that run;
* the packed words: (key - min) << PB | position orders as the (key, position)
  pair whenever the key range is below the limit the kernel tests, and 16-bit
  offsets from the minimum order as the keys.

These pin the layout and arithmetic the kernels rely on; the GPU parity tests
check the kernels themselves against the oracle."""
import random

import pytest


def merge_pair_rev(sk, base, run, IT):
    """Thread `base`'s IT outputs of the pair starting at pb, second run descending."""
    pb = base & ~(2 * run - 1)
    d = base - pb
    lo, hi = max(0, d - run), min(d, run)
    reads = []
    while lo < hi:
        mid = (lo + hi) >> 1
        av = sk[pb + mid]
        bpos = pb + 2 * run - d + mid               # ascending element d-1-mid of the second run
        reads += [pb + mid, bpos]
        bv = sk[bpos]
        if bv < av:
            hi = mid
        else:
            lo = mid + 1
    i, j = pb + lo, pb + 2 * run - 1 - (d - lo)
    reads += [i, j]
    si, sj = sk[i], sk[j]
    out = []
    for k in range(IT):
        tj = sj < si
        out.append(sj if tj else si)
        if k + 1 < IT:
            if tj:
                j -= 1
            else:
                i += 1
            idx = j if tj else i
            reads.append(idx)
            if tj:
                sj = sk[idx]
            else:
                si = sk[idx]
    return out, reads, pb


@pytest.mark.parametrize("run,IT", [(8, 4), (16, 8), (32, 8), (64, 16)])
@pytest.mark.parametrize("values", [4, 50, 10_000])
def test_bitonic_pair_merge(run, IT, values):
    rng = random.Random(run * 1000 + IT * 10 + values)
    for _ in range(40):
        a = sorted(rng.randrange(values) for _ in range(run))
        b = sorted(rng.randrange(values) for _ in range(run))
        if rng.random() < 0.2:                       # one run entirely below the other
            a, b = sorted(a + b)[:run], sorted(a + b)[run:]
        if rng.random() < 0.2:
            a, b = b, a
        sk = a + b[::-1]                              # the layout store_run leaves
        want = sorted(a + b)
        for base in range(0, 2 * run, IT):
            out, reads, pb = merge_pair_rev(sk, base, run, IT)
            assert out == want[base:base + IT]
            assert all(pb <= r < pb + 2 * run for r in reads)


@pytest.mark.parametrize("run,IT", [(64, 64), (2048, 64), (32, 16)])
def test_descending_store_is_the_mirror_of_the_run(run, IT):
    """store_run: a thread of the second run writes its IT sorted elements at
    2 pb + 3 run - 1 - q (q its positions base .. base + IT - 1), which for every
    thread of the run together is the run reversed in place."""
    for pb in (0, 2 * run, 6 * run):
        written = {}
        for base in range(pb + run, pb + 2 * run, IT):
            mb = 2 * pb + 3 * run - base - IT         # the kernel's base for the descending store
            for i in range(IT):
                pos = mb + (IT - 1 - i)
                assert pos == 2 * pb + 3 * run - 1 - (base + i)
                assert pb + run <= pos < pb + 2 * run
                written[pos] = base + i
        assert sorted(written) == list(range(pb + run, pb + 2 * run))
        for pos, q in written.items():
            assert pos - (pb + run) == (pb + 2 * run - 1) - q


@pytest.mark.parametrize("key_bits,pb,word_bits", [(32, 13, 32), (64, 12, 64)])
def test_packed_pair_words_order_as_pairs(key_bits, pb, word_bits):
    """(key - kmin) << PB | position, for leaves whose key range is below
    2^(word_bits - PB) - 1 (the kernel's test), orders exactly as (key, position)
    and never reaches the all-ones padding word."""
    rng = random.Random(key_bits)
    limit = (1 << (word_bits - pb)) - 1
    cap = 1 << pb
    for span in (1, 7, limit // 3, limit - 1):
        kmin = rng.randrange((1 << key_bits) - span)
        n = min(cap, 600)
        keys = [kmin + rng.randrange(span + 1) for _ in range(n)]
        keys[0], keys[-1] = kmin, kmin + span      # the extremes the kernel measures
        assert max(keys) - min(keys) < limit
        words = [((k - kmin) << pb) | p for p, k in enumerate(keys)]
        assert max(words) < (1 << word_bits) - 1
        by_pair = sorted(range(n), key=lambda p: (keys[p], p))
        by_word = sorted(range(n), key=lambda p: words[p])
        assert by_pair == by_word
        # decoding recovers key and position
        for p, w in enumerate(words):
            assert (w >> pb) + kmin == keys[p] and (w & (cap - 1)) == p


def test_narrow_offsets_order_as_keys_and_padding_sorts_last():
    """16-bit offsets from the leaf's minimum (range at most 0xFFFF, minimum at most
    0xFFFF0000): padding 0xFFFF unpacks to kmin + 0xFFFF, no smaller than any key,
    without wrapping past 2^32 - 1."""
    rng = random.Random(5)
    for kmin in (0, 12345, 0x7FFF0000, 0xFFFF0000):
        keys = [kmin + rng.randrange(0x10000) for _ in range(500)]
        keys[0] = kmin
        assert max(keys) - min(keys) <= 0xFFFF
        offs = [k - kmin for k in keys]
        assert all(0 <= o <= 0xFFFF for o in offs)
        assert [kmin + o for o in sorted(offs)] == sorted(keys)
        pad = kmin + 0xFFFF
        assert pad <= 0xFFFFFFFF and pad >= max(keys)
