"""Test-side statement of the batched sort's per-segment rule, written from the
header's contract (not from the library): segment g takes the first class whose
max_len covers its length (the last class when none does); p falls to 1 when
the class has p = 1 or the segment is shorter than 2 p s; the sample seed of
segment g is output g of stream 2 of the SplitMix64 keyed by the batch seed
(computed with the oracle's own generator)."""
from __future__ import annotations

import oracle


def class_of(length: int, classes) -> int:
    for k, c in enumerate(classes):
        if length <= c[0]:
            return k
    return len(classes) - 1


def seg_params(length: int, classes) -> tuple[int, int]:
    _, p, s, _ = classes[class_of(length, classes)]
    if p > 1 and length < 2 * p * s:
        p = 1
    return p, s


def seg_seed(seed: int, g: int) -> int:
    return oracle.splitmix64(seed, 2, g)
