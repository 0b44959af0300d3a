"""Pins for the oracle's k-mismatch search (Section 2: the BWT phase places
each read with at most k mismatches; here all hits on both strands)."""
import numpy as np
import pytest

import oracle
import synth
from tests import golden_cases, refcheck


def _set(res, i):
    return res.as_tuples(i)


@pytest.mark.parametrize("case", golden_cases.cases(), ids=lambda c: f"{c['read']}-k{c['k']}-cap{c['cap']}")
def test_handworked(case):
    g = golden_cases.codes(case["genome"])
    fm = oracle.FMIndex(g)
    b = golden_cases.batch_of(case["read"], case["k"])
    res = fm.align(b, cap=case["cap"])
    assert int(res.total[0]) == case["total"]
    assert _set(res, 0) == case["hits"]
    if case["cap"] == 0:
        bf = oracle.bruteforce(g, b)
        assert _set(bf, 0) == case["hits"]


def _tiny_batches(g, rng, n=60):
    reads, ks = [], []
    for _ in range(n):
        m = int(rng.integers(1, min(40, len(g)) + 1))
        if rng.random() < 0.7:
            p = int(rng.integers(0, len(g) - m + 1))
            r = g[p:p + m].copy()
            if rng.random() < 0.5:
                r = refcheck.rc(r)
            for q in rng.choice(m, size=min(m, int(rng.integers(0, 3))), replace=False):
                r[q] = (r[q] + rng.integers(1, 4)) & 3
        else:
            r = rng.integers(0, 4, m).astype(np.uint8)
        reads.append(r)
        ks.append(int(rng.integers(0, 4)))
    words, off, lens = synth.pack_reads(reads)
    return reads, synth.ReadBatch(words, off, lens, np.array(ks, np.uint8), np.zeros(n, np.int64),
                                  np.zeros(n, np.uint8), np.zeros(n, np.int32))


@pytest.mark.parametrize("kind", ["random", "tandem", "twoletter"])
def test_against_numpy_hamming_scan(kind):
    rng = np.random.default_rng({"random": 1, "tandem": 2, "twoletter": 3}[kind])
    if kind == "random":
        g = rng.integers(0, 4, 3000).astype(np.uint8)
    elif kind == "tandem":
        g = np.resize(np.array([0, 3, 3, 1, 0], np.uint8), 1500)
        g[rng.choice(1500, 20, replace=False)] = rng.integers(0, 4, 20)
    else:
        g = rng.integers(0, 2, 800).astype(np.uint8) * 3       # A/T only
    fm = oracle.FMIndex(g)
    reads, b = _tiny_batches(g, rng)
    res = fm.align(b)
    bf = oracle.bruteforce(g, b)
    for i, r in enumerate(reads):
        want = refcheck.hamming_hits(g, r, int(b.k[i]))
        assert _set(res, i) == want
        assert _set(bf, i) == want
        assert int(res.total[i]) == len(want)


def test_whole_genome_read_and_single_base():
    rng = np.random.default_rng(5)
    g = rng.integers(0, 4, 64).astype(np.uint8)
    fm = oracle.FMIndex(g)
    reads = [g.copy(), g[:1].copy(), refcheck.rc(g)]
    words, off, lens = synth.pack_reads(reads)
    for k in range(4):
        b = synth.ReadBatch(words, off, lens, np.full(3, k, np.uint8), np.zeros(3, np.int64),
                            np.zeros(3, np.uint8), np.zeros(3, np.int32))
        res = fm.align(b)
        for i, r in enumerate(reads):
            assert _set(res, i) == refcheck.hamming_hits(g, r, k)


def test_rejects_bad_input():
    g = np.zeros(10, np.uint8)
    fm = oracle.FMIndex(g)
    for m, k in ((11, 0), (5, 4)):
        words, off, lens = synth.pack_reads([np.zeros(m, np.uint8)])
        b = synth.ReadBatch(words, off, lens, np.array([k], np.uint8), np.zeros(1, np.int64),
                            np.zeros(1, np.uint8), np.zeros(1, np.int32))
        with pytest.raises(ValueError):
            fm.align(b)


def test_empty_batch():
    fm = oracle.FMIndex(np.zeros(10, np.uint8))
    b = synth.ReadBatch(np.zeros(0, np.uint32), np.zeros(1, np.uint64), np.zeros(0, np.uint16),
                        np.zeros(0, np.uint8), np.zeros(0, np.int64), np.zeros(0, np.uint8),
                        np.zeros(0, np.int32))
    res = fm.align(b)
    assert res.total.size == 0 and res.hits.size == 0


@pytest.fixture(scope="module")
def genome_1m():
    g = synth.genome_1m()
    return g, oracle.FMIndex(g.codes, "sais")


def test_slice_against_bruteforce():
    g, b = synth.slice_10k(synth.genome_1m())
    fm = oracle.FMIndex(g.codes, "sort")
    for k in range(4):
        b.k[:] = k
        res = fm.align(b)
        bf = oracle.bruteforce(g.codes, b)
        assert np.array_equal(res.total, bf.total)
        assert np.array_equal(res.offsets, bf.offsets)
        assert np.array_equal(res.hits, bf.hits)


def test_random_genome_ground_truth(genome_1m):
    """On an i.i.d. 1 Mbp genome a 100 bp read has a chance hit with <= 2
    mismatches with probability ~2e6 * 44851 / 4^100, so H(R) is exactly the
    sampled origin with its substitution count."""
    g, fm = genome_1m
    b = synth.reads_1m(g, n=2000)
    res = fm.align(b, cap=1000)
    for i in range(b.n):
        assert _set(res, i) == [(int(b.origin[i]), int(b.strand[i]), int(b.n_subs[i]))]


def test_mismatch_counts_recomputed(genome_1m):
    g, fm = genome_1m
    rng = np.random.default_rng(8)
    b = synth.sample_reads(g, np.full(300, 30), rng.integers(0, 4, 300), rng, subs="count", max_subs=3)
    res = fm.align(b)
    for i in range(b.n):
        r = b.read(i)
        for p, s, d in _set(res, i):
            w = g.codes[p:p + len(r)]
            assert int(((refcheck.rc(r) if s else r) != w).sum()) == d <= b.k[i]


def test_reverse_complement_symmetry(genome_1m):
    g, fm = genome_1m
    rng = np.random.default_rng(9)
    b = synth.sample_reads(g, np.full(200, 24), rng.integers(0, 4, 200), rng, subs="count", max_subs=2)
    words, off, lens = synth.pack_reads([refcheck.rc(b.read(i)) for i in range(b.n)])
    b2 = synth.ReadBatch(words, off, lens, b.k, b.origin, b.strand, b.n_subs)
    r1, r2 = fm.align(b), fm.align(b2)
    for i in range(b.n):
        swapped = sorted((p, 1 - s, d) for p, s, d in _set(r1, i))
        assert _set(r2, i) == swapped


def test_cap_rule_properties():
    """The cap keeps `cap` rows: lowest d first, then + before -, then the
    lexicographically smallest suffixes; total stays exact."""
    g = synth.repeat_genome(6_000, 11, copy_frac=0.0, tandem_frac=0.3,
                            unit_len=(2, 4), array_len=(300, 1000)).codes
    fm = oracle.FMIndex(g, "sort")
    rng = np.random.default_rng(12)
    reads = []
    for _ in range(40):
        p = int(rng.integers(0, len(g) - 16))
        reads.append(g[p:p + 16].copy())
    words, off, lens = synth.pack_reads(reads)
    b = synth.ReadBatch(words, off, lens, rng.integers(0, 3, 40).astype(np.uint8),
                        np.zeros(40, np.int64), np.zeros(40, np.uint8), np.zeros(40, np.int32))
    cap = 25
    full, capped = fm.align(b), fm.align(b, cap=cap)
    # suffix ranks by sorting suffix byte strings (independent of the oracle's SA)
    t = (g + 1).tobytes() + b"\x00"
    order = sorted(range(len(t)), key=lambda i: t[i:])
    suffix_rank = np.empty(len(t), np.int64)
    suffix_rank[order] = np.arange(len(t))
    n_capped = 0
    for i in range(b.n):
        allh, kept = _set(full, i), _set(capped, i)
        assert int(capped.total[i]) == int(full.total[i]) == len(allh)
        assert len(kept) == min(cap, len(allh))
        assert set(kept) <= set(allh)
        if len(allh) <= cap:
            continue
        n_capped += 1
        key = lambda h: (h[2], h[1], suffix_rank[h[0]])
        dropped = set(allh) - set(kept)
        assert max(key(h) for h in kept) < min(key(h) for h in dropped)
    assert n_capped > 5


def test_cap_order_by_suffix_comparison():
    """Suffix ranks in the cap rule, checked by direct string comparison."""
    g = np.resize(np.array([0, 3], np.uint8), 400)        # (AT)^200
    fm = oracle.FMIndex(g, "sort")
    b = golden_cases.batch_of("ATATATAT", 0)
    res = fm.align(b, cap=10)
    kept = [p for p, s, d in _set(res, 0)]
    allh = refcheck.hamming_hits(g, golden_cases.codes("ATATATAT"), 0)
    tail = lambda p: tuple(g[p:].tolist()) + (-1,)
    plus = sorted((p for p, s, d in allh if s == 0), key=tail)
    assert sorted(kept) == sorted(plus[:10])
    assert int(res.total[0]) == len(allh)


@pytest.mark.parametrize("kind", ["random", "tandem"])
def test_best_stratum_against_numpy_scan(kind):
    """Best-stratum reporting = the Hamming hits with the read's smallest d
    (numpy scan filtered by its definition)."""
    rng = np.random.default_rng({"random": 21, "tandem": 22}[kind])
    if kind == "random":
        g = rng.integers(0, 4, 3000).astype(np.uint8)
    else:
        g = np.resize(np.array([0, 3, 3, 1, 0], np.uint8), 1500)
        g[rng.choice(1500, 20, replace=False)] = rng.integers(0, 4, 20)
    fm = oracle.FMIndex(g)
    reads, b = _tiny_batches(g, rng)
    res = fm.align_best_stratum(b)
    for i, r in enumerate(reads):
        allh = refcheck.hamming_hits(g, r, int(b.k[i]))
        if allh:
            dmin = min(d for _, _, d in allh)
            allh = [h for h in allh if h[2] == dmin]
        assert _set(res, i) == allh
        assert int(res.total[i]) == len(allh)


def test_best_stratum_cap_order_by_suffix_comparison():
    """Over the cap, best-stratum keeps the first rows by (strand, suffix)."""
    g = synth.repeat_genome(6_000, 11, copy_frac=0.0, tandem_frac=0.3,
                            unit_len=(2, 4), array_len=(300, 1000)).codes
    fm = oracle.FMIndex(g, "sort")
    rng = np.random.default_rng(13)
    reads = []
    for _ in range(40):
        p = int(rng.integers(0, len(g) - 16))
        reads.append(g[p:p + 16].copy())
    words, off, lens = synth.pack_reads(reads)
    b = synth.ReadBatch(words, off, lens, rng.integers(0, 3, 40).astype(np.uint8),
                        np.zeros(40, np.int64), np.zeros(40, np.uint8), np.zeros(40, np.int32))
    cap = 7
    full, capped = fm.align_best_stratum(b), fm.align_best_stratum(b, cap=cap)
    t = (g + 1).tobytes() + b"\x00"
    order = sorted(range(len(t)), key=lambda i: t[i:])
    suffix_rank = np.empty(len(t), np.int64)
    suffix_rank[order] = np.arange(len(t))
    n_capped = 0
    for i in range(b.n):
        allh, kept = _set(full, i), _set(capped, i)
        assert int(capped.total[i]) == int(full.total[i]) == len(allh)
        assert len({d for _, _, d in allh}) <= 1
        assert len(kept) == min(cap, len(allh)) and set(kept) <= set(allh)
        if len(allh) > cap:
            n_capped += 1
            key = lambda h: (h[1], suffix_rank[h[0]])
            dropped = set(allh) - set(kept)
            assert max(key(h) for h in kept) < min(key(h) for h in dropped)
    assert n_capped > 5
