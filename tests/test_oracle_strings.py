"""Pins of the oracle's 32-byte string keys (the paper's workload: random
32-byte strings compared with memcmp, Section 3), against facts outside it:
Python's own bytes order (memcmp semantics, unsigned bytes), numpy's stable
lexsort over the byte columns (brute force), splitters recomputed by sorting
the whole sample with lexsort, bucket sizes counted against those splitters,
and the Lemma 1 bound for SqDet."""
import numpy as np
import pytest

import oracle
from paper_1608_08648_gb300 import inputs
from tests import refcheck as rc


def lex_perm(keys: np.ndarray, tags: np.ndarray | None = None) -> np.ndarray:
    """Stable order of (32 bytes, tag) rows: lexsort with the first byte most significant."""
    cols = [keys[:, k] for k in range(31, -1, -1)]
    if tags is not None:
        cols = [tags] + cols
    return np.lexsort(cols)


def test_str_cmp_is_unsigned_memcmp():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        a = rng.integers(0, 256, 32, dtype=np.uint8)
        b = a.copy()
        k = rng.integers(0, 32)
        b[k:] = rng.integers(0, 256, 32 - k, dtype=np.uint8)
        ab, bb = a.tobytes(), b.tobytes()
        assert oracle.str_cmp(ab, bb) == (ab > bb) - (ab < bb)
    assert oracle.str_cmp(b"\x80" + bytes(31), b"\x7f" + b"\xff" * 31) == 1   # bytes are unsigned


@pytest.mark.parametrize("dist", list(inputs.STR_DISTRIBUTIONS))
@pytest.mark.parametrize("split", ["ran", "det"])
def test_strings_vs_brute_force(dist, split):
    n = 6007
    keys = inputs.strings(dist, n, seed=4).numpy()
    vals = np.arange(n, dtype=np.uint32)
    r = oracle.sort(keys, "s32", split, 16, 4, seed=9, vals=vals)
    perm = lex_perm(keys)
    assert np.array_equal(r["keys"], keys[perm])
    assert np.array_equal(r["vals"], vals[perm]), "payload not in stable order"
    assert int(r["bucket_sizes"].sum()) == n


def ran_splitters(keys, p, s, seed):
    m = p * s - 1
    pos = rc.ran_sample_positions(seed, m, len(keys))
    order = lex_perm(keys[pos], pos)
    pick = [order[i * s - 1] for i in range(1, p)]
    return pos[pick], pos[pick]


def det_splitters(keys, p, r):
    n = len(keys)
    cs = rc.chunk_bounds(n, p)
    m = r * p
    elem, tag = [], []
    for k in range(p):
        a, b = cs[k], cs[k + 1]
        perm = a + lex_perm(keys[a:b])
        c = b - a
        for j in range(1, m + 1):
            loc = -(-j * c // m) - 1
            elem.append(perm[loc])
            tag.append(a + loc)
    elem, tag = np.array(elem), np.array(tag)
    order = lex_perm(keys[elem], tag)
    pick = [order[i * m - 1] for i in range(1, p)]
    return elem[pick], tag[pick]


def bucket_sizes(keys, tags, spl_keys, spl_tags, p):
    """Count, for every element, the splitters strictly below it in (bytes, tag) order."""
    sizes = np.zeros(p, dtype=np.int64)
    sk = [bytes(x) for x in spl_keys]
    for row, t in zip(keys, tags):
        kb = bytes(row)
        b = sum(1 for s, st in zip(sk, spl_tags) if (s, st) < (kb, t))
        sizes[b] += 1
    return sizes


@pytest.mark.parametrize("dist", ["uniform", "dup", "ties16"])
def test_ran_splitters_and_buckets_recomputed(dist):
    n, p, s, seed = 3001, 8, 6, 11
    keys = inputs.strings(dist, n, seed=6).numpy()
    r = oracle.sort(keys, "s32", "ran", p, s, seed=seed, merge=False)
    elem, tag = ran_splitters(keys, p, s, seed)
    assert np.array_equal(r["spl_keys"], keys[elem])
    assert np.array_equal(r["spl_tags"].astype(np.int64), tag)
    sizes = bucket_sizes(keys, np.arange(n), keys[elem], tag, p)
    assert np.array_equal(r["bucket_sizes"].astype(np.int64), sizes)


@pytest.mark.parametrize("dist", ["uniform", "dup", "prefix24"])
def test_det_splitters_buckets_and_lemma1(dist):
    n, p, r_ = 4096, 8, 2
    keys = inputs.strings(dist, n, seed=7).numpy()
    r = oracle.sort(keys, "s32", "det", p, r_, seed=0, merge=False)
    elem, tag = det_splitters(keys, p, r_)
    assert np.array_equal(r["spl_keys"], keys[elem])
    assert np.array_equal(r["spl_tags"].astype(np.int64), tag)
    # tags of every element: its position among the stably sorted sequences
    cs = rc.chunk_bounds(n, p)
    tags = np.empty(n, dtype=np.int64)
    for k in range(p):
        a, b = cs[k], cs[k + 1]
        tags[a + lex_perm(keys[a:b])] = a + np.arange(b - a)
    sizes = bucket_sizes(keys, tags, keys[elem], tag, p)
    assert np.array_equal(r["bucket_sizes"].astype(np.int64), sizes)
    assert int(r["bucket_sizes"].max()) <= rc.derived_det_bound(n, p, r_)
