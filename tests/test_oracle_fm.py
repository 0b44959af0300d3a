"""Pins for the oracle's plain FM index (BWT, C, Occ, exact backward search)."""
import numpy as np
import pytest

import oracle
import synth
from tests import refcheck


@pytest.fixture(scope="module")
def small():
    g = synth.repeat_genome(50_000, 9, copy_frac=0.1, copy_len=(300, 2000),
                            tandem_frac=0.05, array_len=(100, 1000)).codes
    return g, oracle.FMIndex(g, "sort")


def test_bwt_matches_definition(small):
    g, fm = small
    sa = fm.sa()
    t = np.concatenate([g, [4]]).astype(np.uint8)          # $ = 4 in BWT coding
    want = np.where(sa == 0, 4, t[(sa.astype(np.int64) - 1) % len(t)])
    assert np.array_equal(fm.bwt(), want)


def test_C_and_occ_against_cumulative_counts(small):
    g, fm = small
    bwt = fm.bwt()
    counts = np.bincount(g, minlength=4)
    assert [fm.C(c) for c in range(4)] == [1 + int(counts[:c].sum()) for c in range(4)]
    rng = np.random.default_rng(1)
    rows = np.concatenate([rng.integers(0, fm.rows + 1, 300), [0, 1, 63, 64, 65, fm.rows - 1, fm.rows]])
    for c in range(4):
        cum = np.concatenate([[0], np.cumsum(bwt == c)])
        for i in rows:
            assert fm.occ(c, int(i)) == int(cum[i])
    # column sums: every row is one of A, C, G, T or the single $
    assert sum(fm.occ(c, fm.rows) for c in range(4)) + 1 == fm.rows


def test_lf_consistency(small):
    g, fm = small
    sa = fm.sa().astype(np.int64)
    bwt = fm.bwt()
    rng = np.random.default_rng(2)
    for j in rng.integers(0, fm.rows, 2000):
        c = int(bwt[j])
        if c == 4:
            assert sa[j] == 0
            continue
        lf = fm.C(c) + fm.occ(c, int(j))
        assert sa[lf] == sa[j] - 1


def test_exact_interval_size_is_occurrence_count(small):
    g, fm = small
    rng = np.random.default_rng(4)
    for m in range(1, 21):
        for _ in range(10):
            if rng.random() < 0.5:       # pattern present in G
                p0 = int(rng.integers(0, len(g) - m + 1))
                p = g[p0:p0 + m].copy()
            else:
                p = rng.integers(0, 4, m).astype(np.uint8)
            l, r = fm.exact_interval(p)
            assert r - l == refcheck.count_occurrences(g, p)
            # and every row of the interval starts with p
            sa = fm.sa()
            for j in range(l, min(r, l + 5)):
                assert np.array_equal(g[sa[j]:sa[j] + m], p)
