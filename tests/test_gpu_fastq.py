"""FASTQ to SAM through the GPU: reads with ambiguous bases from FASTQ files,
searched on the GPU, recounted by the N rule, paired on the GPU and written
as SAM; each step equals the oracle's (bit-exact lists, byte-identical SAM)."""
import numpy as np
import pytest

import oracle
import synth
from tests import gpu_common as gc
from tests import samcheck

pytestmark = pytest.mark.gpu

WINDOW = (200, 600)


@pytest.fixture(scope="module")
def setup():
    m = gc.mica()
    g = synth.uniform_genome(30_000, synth.SEED_FASTQ + 10).codes
    ref = m.Reference.create(synth.to_acgt_bytes(g), [len(g)], ["chrS"])
    return m, g, ref, m.Index.build(ref), oracle.FMIndex(g)


def _records(b):
    return [(n, q, list(a), int(k)) for (n, q, a), k in zip((b.record(i) for i in range(b.n)), b.k)]


def test_single_reads(setup, tmp_path):
    m, g, ref, idx, fm = setup
    rng = np.random.Generator(np.random.PCG64(synth.SEED_FASTQ + 11))
    n = 3000
    reads = synth.sample_reads(synth.Genome(g), rng.choice(np.array([50, 100, 150]), size=n),
                               np.full(n, 2, np.uint8), rng, subs="count", max_subs=2)
    (text,), amb, _ = synth.to_fastq(reads, n_frac=0.4, max_n=2)
    path = tmp_path / "r.fq"
    path.write_bytes(text)
    with m.FastqReader(str(path)) as fq:
        (b,) = list(fq.batches(10_000))
    got = idx.align_batch(b, hit_cap=0)
    want = fm.align(b)
    gc.assert_same(got, want, "search")
    fgot, dgot = b.filter_n(ref, got)
    fwant, dwant = oracle.n_filter(want, [b.read(i) for i in range(b.n)], amb, b.k, g)
    assert dgot == dwant > 0
    gc.assert_same(fgot, fwant, "N rule")
    sam = tmp_path / "r.sam"
    with m.SamWriter(str(sam), ref, secondary=True) as w:
        w.write_batch(b, got)
    expect = samcheck.sam_text(["chrS"], [0, len(g)], [], synth.to_acgt_bytes(g).decode(), b, want,
                               secondary=True, records=_records(b))
    assert open(sam).read() == expect


def test_paired_reads(setup, tmp_path):
    m, g, ref, idx, fm = setup
    pairs = synth.paired_reads(g, 1000, seed=synth.SEED_FASTQ + 12, m=100, insert_mean=350.0, insert_sd=40.0)
    texts, amb, _ = synth.to_fastq(pairs, mate_suffix=True, n_frac=0.3)
    paths = []
    for j, t in enumerate(texts):
        p = tmp_path / f"p{j + 1}.fq"
        p.write_bytes(t)
        paths.append(str(p))
    with m.FastqReader(*paths) as fq:
        (b,) = list(fq.batches(10_000))
    got, _ = b.filter_n(ref, idx.align_batch(b, hit_cap=0))
    want, _ = oracle.n_filter(fm.align(b), [b.read(i) for i in range(b.n)], amb, b.k, g)
    gc.assert_same(got, want, "paired N rule")
    pr = m.pair_batch(got, b.lengths, *WINDOW)
    opr = samcheck.pairs_array(oracle.pair(want, b.lengths, *WINDOW), m.PAIR_DTYPE)
    assert (pr == opr).all()
    sam = tmp_path / "p.sam"
    with m.SamWriter(str(sam), ref) as w:
        w.write_batch(b, got, pr)
    expect = samcheck.sam_text(["chrS"], [0, len(g)], [], synth.to_acgt_bytes(g).decode(), b, want, opr,
                               records=_records(b))
    assert open(sam).read() == expect
