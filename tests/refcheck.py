"""Independent numpy checks used to pin the oracle and to check the CUDA path.

Nothing here is shared with the oracle or with the library: the key order is
taken from the textbook order-preserving integer maps (sign flip for int32,
IEEE 754 totalOrder bit map for float64) and every selection is done with
numpy's own stable sorts and lexsort.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_1608_08648_gb300 import inputs

NP_DT = {"i32": np.int32, "u64": np.uint64, "f64": np.float64}
MASK64 = (1 << 64) - 1


def order_key(keys: np.ndarray, kt: str) -> np.ndarray:
    """A uint64 array whose unsigned order is the key order (f64: totalOrder)."""
    if kt == "i32":
        return (keys.astype(np.int64) + (1 << 31)).astype(np.uint64)
    if kt == "u64":
        return keys.astype(np.uint64)
    bits = keys.view(np.uint64)
    neg = (bits >> np.uint64(63)) != 0
    return np.where(neg, ~bits, bits | np.uint64(1 << 63))


def brute_perm(keys: np.ndarray, kt: str) -> np.ndarray:
    """Stable sorting permutation of the keys (the output order of a stable sort)."""
    return np.argsort(order_key(keys, kt), kind="stable")


def chunk_bounds(n: int, p: int) -> np.ndarray:
    return np.array([(k * n) // p for k in range(p + 1)], dtype=np.int64)


def det_tags(keys: np.ndarray, kt: str, p: int) -> np.ndarray:
    """Tag of every original element for SqDet: its position in the concatenation of
    the p stably sorted sequences (the flattened (sequence, local index) tag)."""
    ok = order_key(keys, kt)
    cs = chunk_bounds(len(keys), p)
    tags = np.empty(len(keys), dtype=np.int64)
    for k in range(p):
        a, b = cs[k], cs[k + 1]
        perm = np.argsort(ok[a:b], kind="stable")
        tags[a + perm] = a + np.arange(b - a)
    return tags


def ran_sample_positions(seed: int, m: int, n: int) -> np.ndarray:
    """floor(u_j * n / 2^64) for j < m, with u_j from stream 1 (the generator module's
    SplitMix64 implementation, independent of the oracle's)."""
    u = inputs.u64(seed, 1, torch.arange(m, dtype=torch.int64)).numpy().view(np.uint64)
    return np.array([(int(x) * n) >> 64 for x in u], dtype=np.int64)


def splitters(keys: np.ndarray, kt: str, split: str, p: int, s: int, seed: int):
    """(original element index, tag) of each of the p-1 splitters, computed by sorting
    the whole sample with lexsort and indexing it (no merging)."""
    n = len(keys)
    ok = order_key(keys, kt)
    if split == "det":
        tags = det_tags(keys, kt, p)
        cs = chunk_bounds(n, p)
        m = s * p
        elem = []
        for k in range(p):
            a, b = cs[k], cs[k + 1]
            perm = a + np.argsort(ok[a:b], kind="stable")
            c = b - a
            for j in range(1, m + 1):
                elem.append(perm[-(-j * c // m) - 1])
        elem = np.array(elem, dtype=np.int64)
        stag = tags[elem]
        stride = m
    else:
        elem = ran_sample_positions(seed, p * s - 1, n)
        stag = elem.copy()
        stride = s
    order = np.lexsort((stag, ok[elem]))
    pick = [order[i * stride - 1] for i in range(1, p)]
    return elem[pick], stag[pick]


def bucket_of(keys: np.ndarray, kt: str, tags: np.ndarray, spl_elem: np.ndarray,
              spl_tag: np.ndarray) -> np.ndarray:
    """Bucket of every element: the number of splitters strictly below it in the
    tagged (key, tag) order."""
    ok = order_key(keys, kt)
    sok = ok[spl_elem]
    lo = np.searchsorted(sok, ok, side="left")
    hi = np.searchsorted(sok, ok, side="right")
    b = lo.astype(np.int64)
    for i in np.nonzero(hi > lo)[0]:
        b[i] += int(np.sum(spl_tag[lo[i]:hi[i]] < tags[i]))
    return b


def derived_det_bound(n: int, p: int, s: int) -> int:
    """Bucket-size bound of the Lemma 1 argument without padding: with q = p
    sequences of m = s p segments each, x_min the smallest segment and
    sigma = ceil(|T|/p), every bucket holds at most n - x_min (q m - q + 1 - sigma)."""
    cs = chunk_bounds(n, p)
    m = s * p
    x_min = min(int(cs[k + 1] - cs[k]) // m for k in range(p))
    sigma = -(-(p * m) // p)
    return n - x_min * (p * m - p + 1 - sigma)
