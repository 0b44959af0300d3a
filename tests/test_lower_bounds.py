"""Pins of the mismatch lower bound the pruned search uses (Li and Durbin's
D array, written from its definition in tests/refcheck.py): the bound never
exceeds the true minimum number of substitutions of a pattern prefix against
any genome window (brute force), it is zero for patterns taken from the
genome, and it counts planted absent pieces."""
import numpy as np

from tests import refcheck


def _d(bps, i):
    return sum(b <= i for b in bps)


def test_bound_never_exceeds_the_brute_force_minimum():
    rng = np.random.default_rng(3)
    g = rng.integers(0, 4, 3_000).astype(np.uint8)
    for trial in range(40):
        m = int(rng.integers(14, 60))
        if trial % 2:
            o = int(rng.integers(0, g.size - m))
            p = g[o:o + m].copy()
            flip = rng.choice(m, size=int(rng.integers(0, 5)), replace=False)
            p[flip] = (p[flip] + rng.integers(1, 4, size=flip.size)) & 3
        else:
            p = rng.integers(0, 4, m).astype(np.uint8)
        bps = refcheck.lower_bound_breakpoints(g, p, 3, 12)
        assert bps == sorted(bps) and len(bps) <= 4
        for i in range(0, m - min(m, 12) + 1):
            assert _d(bps, i) <= refcheck.min_prefix_mismatches(g, p, i)


def test_bound_is_zero_on_genome_substrings_and_counts_absent_pieces():
    rng = np.random.default_rng(4)
    g = rng.integers(0, 3, 5_000).astype(np.uint8)      # no T in the genome
    p = g[100:160].copy()
    assert refcheck.lower_bound_breakpoints(g, p, 3, 12) == []
    # every T is a piece of its own that cannot occur
    p[[5, 20, 33]] = 3
    assert refcheck.lower_bound_breakpoints(g, p, 3, 12) == [6, 21, 34]
    assert refcheck.lower_bound_breakpoints(g, p, 1, 12) == [6, 21]
    # positions inside the seed window (the last q bases) are not scanned
    p2 = g[100:160].copy()
    p2[55] = 3
    assert refcheck.lower_bound_breakpoints(g, p2, 3, 12) == []


def test_word_packing():
    assert refcheck.lb_word([]) == (1 << 64) - 1
    v = refcheck.lb_word([6, 21, 34])
    assert v & 511 == 6 and (v >> 9) & 511 == 21 and (v >> 18) & 511 == 34 and (v >> 27) & 511 == 511
