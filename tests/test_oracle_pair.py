"""Pins of the oracle's mate pairing: hand-worked cases and the generator's
true fragments on a random genome, where chance hits of 150 bp mates with
k <= 2 are vanishingly rare, so each pair's only concordant placement is its
true fragment with the mates' true substitution counts."""
import numpy as np

import oracle
import synth


class _Hits:
    """A result stub: offsets plus per-read (pos, strand, mm) lists."""

    def __init__(self, lists):
        self.lists = lists
        self.offsets = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.uint64)

    def as_tuples(self, i):
        return sorted(self.lists[i])


def test_handworked_pairs():
    m = [150, 150, 150, 150, 100, 150]
    r = _Hits([
        # pair 0: one concordant combination (mate 1 +, mate 2 -, fragment 430)
        [(100, 0, 1), (500, 1, 0)], [(380, 0, 2), (380, 1, 0), (900, 1, 1)],
        # pair 1: mate 2 on +, two partners of mate 1 (fragments 300 and 700) with equal mm
        [(1000, 1, 1), (1400, 1, 0)], [(850, 0, 1), (600, 0, 2)],
        # pair 2: same strands only -> not paired
        [(10, 0, 0)], [(200, 0, 0)],
    ])
    got = oracle.pair(r, m, 300, 700)
    assert got[0] == (1, 1, 100, 380, 0, 1)
    # pair 1: + hits of mate 2: 850 (mm 1) and 600 (mm 2); - hits of mate 1 (m = 150)
    #   850 with 1000: L = 1000 + 150 - 850 = 300 (mm 2); 850 with 1400: L = 700 (mm 1)
    #   600 with 1000: L = 550 (mm 3);                    600 with 1400: L = 950 (out)
    assert got[1] == (3, 1, 850, 1400, 1, 1)
    assert got[2] == (0, 0, 0, 0, 0, 0)
    # the window bounds are inclusive; a narrower window drops the 300 and 700 fragments
    assert oracle.pair(r, m, 301, 699)[1] == (1, 1, 600, 1000, 1, 3)


def test_true_fragments_on_a_random_genome():
    g = synth.uniform_genome(300_000, 77)
    b = synth.paired_reads(g.codes, 150, seed=78)
    res = oracle.FMIndex(g.codes, "sort").align(b, cap=1000)
    pairs = oracle.pair(res, b.lengths, 300, 700)
    for p, got in enumerate(pairs):
        i1, i2 = 2 * p, 2 * p + 1
        if b.n_subs[i1] > 2 or b.n_subs[i2] > 2:
            assert got[0] == 0
            continue
        plus = i1 if b.strand[i1] == 0 else i2
        minus = i2 if plus == i1 else i1
        frag = int(b.origin[minus]) + 150 - int(b.origin[plus])
        assert 300 <= frag <= 700
        assert got == (1, 1, int(b.origin[plus]), int(b.origin[minus]), 0 if plus == i1 else 1,
                       int(b.n_subs[i1] + b.n_subs[i2]))
