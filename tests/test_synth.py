"""Pins of the synthetic input generators (the workloads' recipe): read
content against the genome and the recorded origin/strand/substitutions,
length and budget mixes, paired-end geometry, the human-scale composition
and the serving request sizes.  Small sizes only: CPU, seconds."""
import numpy as np

import synth
from tests import refcheck


def _mismatches(g, b, i):
    r = b.read(i)
    o, m = int(b.origin[i]), int(b.lengths[i])
    w = g[o:o + m]
    return int(((refcheck.rc(r) if b.strand[i] else r) != w).sum())


def test_packing_round_trip():
    rng = np.random.default_rng(1)
    reads = [rng.integers(0, 4, int(m)).astype(np.uint8) for m in (1, 15, 16, 17, 150, 256)]
    words, off, lens = synth.pack_reads(reads)
    b = synth.ReadBatch(words, off, lens, np.zeros(6, np.uint8), np.zeros(6, np.int64), np.zeros(6, np.uint8),
                        np.zeros(6, np.int32))
    for i, r in enumerate(reads):
        assert np.array_equal(b.read(i), r)
    sub = b.subset([5, 0, 3])
    for j, i in enumerate((5, 0, 3)):
        assert np.array_equal(sub.read(j), reads[i])


def test_uneven_reads_match_their_origins():
    g = synth.repeat_genome(400_000, 5)
    b = synth.sample_reads(g, np.asarray(synth.UNEVEN_LENGTHS)[np.arange(400) % 4], np.arange(400) % 4,
                           np.random.default_rng(6), subs="rate", sub_rate=0.01, repeat_frac=0.3)
    assert set(np.unique(b.lengths)) == set(synth.UNEVEN_LENGTHS)
    for i in range(b.n):
        assert _mismatches(g.codes, b, i) == int(b.n_subs[i])
    # about 30% of the origins inside planted regions (plus the uniform ones that land there)
    inside = 0
    for i in range(b.n):
        o = int(b.origin[i])
        inside += any(s <= o < e for s, e, _ in g.regions)
    assert 0.25 < inside / b.n < 0.6


def test_repeat_genome_fractions():
    n = 2_000_000
    g = synth.repeat_genome(n, 9)
    copies = sum(e - s for s, e, k in g.regions if k == "copy")
    tandem = sum(e - s for s, e, k in g.regions if k == "tandem")
    assert 0.05 * n <= copies < 0.05 * n + 10_001
    assert 0.01 * n <= tandem < 0.01 * n + 5_001


def test_paired_reads_geometry_and_errors():
    g = synth.uniform_genome(500_000, 3).codes
    b = synth.paired_reads(g, 300, seed=4)
    assert b.n == 600 and np.all(b.lengths == 150)
    for p in range(300):
        i1, i2 = 2 * p, 2 * p + 1
        assert int(b.strand[i1]) != int(b.strand[i2])
        plus = i1 if b.strand[i1] == 0 else i2
        minus = i2 if plus == i1 else i1
        frag = int(b.origin[minus]) + 150 - int(b.origin[plus])
        assert 300 <= frag <= 700
        for i in (i1, i2):
            assert _mismatches(g, b, i) == int(b.n_subs[i])
    # 1% i.i.d. errors over 150 bases: mean 1.5 per mate
    assert 1.2 < float(np.mean(b.n_subs)) < 1.8


def test_human_genome_composition_small():
    g = synth.human_genome(4_000_000, seed=123)
    n = g.n
    cover = np.zeros(n, bool)
    kinds = {}
    for s, e, k in g.regions:
        cover[s:e] = True
        kinds[k] = kinds.get(k, 0) + (e - s)
    # planted lengths: 15% + 25% + 5% of n (before overlaps); covered share about 45% less overlaps
    assert abs(kinds["fam300"] / n - 0.15) < 0.01
    assert abs(kinds["fam6k"] / n - 0.25) < 0.01
    assert 0.05 <= kinds["tandem"] / n < 0.06
    assert 0.33 < cover.mean() < 0.46
    d = synth.donor_of(g, seed=124)
    snv = float(np.mean(d != g.codes))
    assert 0.0008 < snv < 0.0011


def test_serve_requests():
    d = synth.uniform_genome(200_000, 8).codes
    reqs = synth.serve_requests(d, 40, seed=9, size_range=(100, 10_000))
    sizes = np.array([r.n for r in reqs])
    assert sizes.min() >= 100 and sizes.max() <= 10_000
    # log-uniform: about half the requests below the geometric mean 1,000
    assert 0.3 < np.mean(sizes < 1_000) < 0.7
    lens = np.concatenate([r.lengths for r in reqs])
    ks = np.concatenate([r.k for r in reqs])
    assert set(np.unique(lens)) == {100, 150, 250}
    assert set(np.unique(ks)) == {0, 1, 2}
    r = reqs[0]
    for i in range(min(r.n, 50)):
        assert _mismatches(d, r, i) == int(r.n_subs[i])
