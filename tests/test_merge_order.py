"""Pin of the reading behind the split + merge organisation of SqDet (Algorithm 1,
step 5, OS_DET_MERGE): a bucket's p pieces (piece k from sorted sequence k, its
elements tagged start_k + local index) merged by ceil(log2 p) passes of pairwise
merges -- pass l merges runs of 2^(l-1) consecutive pieces in pairs, the left run
winning ties -- give exactly the tagged order of Section 2.2, i.e. the sort by
(key, tag).  Checked for p that are not powers of two (odd runs) and heavy ties."""
import numpy as np
import pytest


def pairwise_passes(pieces, left_wins=True):
    runs = [list(pc) for pc in pieces]
    while len(runs) > 1:
        nxt = []
        for i in range(0, len(runs), 2):
            if i + 1 == len(runs):
                nxt.append(runs[i])             # odd run: carried to the next pass
                continue
            a, b, out = runs[i], runs[i + 1], []
            ia = ib = 0
            while ia < len(a) or ib < len(b):
                if left_wins:
                    take_b = ia == len(a) or (ib < len(b) and b[ib][0] < a[ia][0])   # ties: left run
                else:
                    take_b = ia == len(a) or (ib < len(b) and b[ib][0] <= a[ia][0])
                out.append(b[ib] if take_b else a[ia])
                ib += take_b
                ia += not take_b
            nxt.append(out)
        runs = nxt
    return runs[0] if runs else []


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 13, 64, 100])
@pytest.mark.parametrize("distinct", [2, 7, 1000])
def test_pairwise_left_first_is_tagged_order(p, distinct):
    rng = np.random.default_rng(p * 1000 + distinct)
    pieces, start = [], 0
    for k in range(p):
        c = int(rng.integers(0, 40))
        keys = np.sort(rng.integers(0, distinct, c))
        pieces.append([(int(x), start + l) for l, x in enumerate(keys)])   # tag = start_k + l
        start += c + int(rng.integers(0, 5))                               # sequences in order
    merged = pairwise_passes(pieces)
    expect = sorted((e for pc in pieces for e in pc), key=lambda e: (e[0], e[1]))
    assert merged == expect


def test_right_first_would_break_the_tagged_order():
    # the same passes taking the right run on ties give another order: the rule matters
    pieces = [[(1, 0), (1, 1)], [(1, 10)]]
    assert [t for _, t in pairwise_passes(pieces)] == [0, 1, 10]
    assert [t for _, t in pairwise_passes(pieces, left_wins=False)] == [10, 0, 1]
