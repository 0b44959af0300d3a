"""A reference of several contigs with ambiguous bases, end to end on the GPU:
index built from the reference text, reads searched and mates paired by the
CUDA path, hits filtered to placements on the reference and written as SAM.
Every step equals the oracle's (bit-exact hit lists, byte-identical SAM)."""
import numpy as np
import pytest

import oracle
import synth
from tests import gpu_common as gc
from tests import samcheck

pytestmark = pytest.mark.gpu

NAMES = ["chr1", "chr2", "chrUn_1", "chrM"]
WINDOW = (200, 600)


@pytest.fixture(scope="module")
def setup():
    m = gc.mica()
    contigs = synth.multi_contig_reference()
    g, starts, runs = oracle.reference_concat(contigs)
    ref = m.Reference.create(b"".join(contigs), [len(c) for c in contigs], NAMES)
    assert ref.text() == synth.to_acgt_bytes(g)
    return m, contigs, g, starts, runs, ref, m.Index.build(ref), oracle.FMIndex(g)


def _single(g, starts, runs):
    rng = np.random.Generator(np.random.PCG64(synth.SEED_REFERENCE_READS + 3))
    regions = [(max(0, s - 160), min(len(g), s + 160), "boundary") for s in starts[1:-1]]
    regions += [(max(0, s - 160), min(len(g), e + 160), "ambiguous") for s, e in runs]
    n = 2000
    lengths = rng.choice(np.array([40, 100, 150, 250]), size=n)
    k = rng.integers(0, 4, size=n, dtype=np.uint8)
    return synth.sample_reads(synth.Genome(g, regions), lengths, k, rng, subs="count", max_subs=3,
                              repeat_frac=0.5)


@pytest.mark.parametrize("cap,report", [(0, "all"), (3, "all"), (2, "best_stratum")])
def test_filtered_search_and_sam_equal_oracle(setup, tmp_path, cap, report):
    m, contigs, g, starts, runs, ref, idx, fm = setup
    reads = _single(g, starts, runs)
    got = idx.align_batch(reads, hit_cap=cap, report=report)
    want = fm.align(reads, cap=cap) if report == "all" else fm.align_best_stratum(reads, cap=cap)
    gc.assert_same(got, want, "unfiltered")
    fgot, dgot = ref.filter(got, reads.lengths)
    fwant, dwant = oracle.reference_filter(want, reads.lengths, starts, runs)
    assert dgot == dwant > 0
    gc.assert_same(fgot, fwant, "filtered")
    path = tmp_path / "gpu.sam"
    with m.SamWriter(str(path), ref, secondary=True) as w:
        w.write(reads, got)
    text = samcheck.sam_text(NAMES, starts, runs, synth.to_acgt_bytes(g).decode(), reads, want, secondary=True)
    assert open(path).read() == text


def test_paired_sam_equals_oracle(setup, tmp_path):
    m, contigs, g, starts, runs, ref, idx, fm = setup
    reads = synth.paired_reads(g, 1000, seed=synth.SEED_REFERENCE_READS + 4, m=100, insert_mean=350.0,
                               insert_sd=40.0)
    got = idx.align_batch(reads, hit_cap=0)
    want = fm.align(reads)
    gc.assert_same(got, want, "paired")
    pairs = m.pair_batch(got, reads.lengths, *WINDOW)
    opairs = samcheck.pairs_array(oracle.pair(want, reads.lengths, *WINDOW), m.PAIR_DTYPE)
    assert (pairs == opairs).all()
    path = tmp_path / "gpu_pairs.sam"
    with m.SamWriter(str(path), ref) as w:
        w.write(reads, got, pairs)
    text = samcheck.sam_text(NAMES, starts, runs, synth.to_acgt_bytes(g).decode(), reads, want, opairs)
    assert open(path).read() == text
