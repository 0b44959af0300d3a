"""The pruned search (mismatch lower bounds from the reversed genome's
occurrence blocks) through the C ABI: the GPU's lower-bound words equal the
definition in tests/refcheck.py, and pruning changes the work, never the
result -- pruned = unpruned = oracle for every kernel."""
import numpy as np
import pytest

import oracle
import synth
from tests import gpu_common as gc
from tests import refcheck

pytestmark = pytest.mark.gpu

KERNELS = ("persistent", "plain", "plain_by_length")


def _reads_from(g, rng, n):
    reads, ks = [], []
    for t in range(n):
        m = int(rng.choice([5, 11, 12, 13, 30, 64, 100, 150, 200, 256]))
        if t % 3 == 2:
            r = rng.integers(0, 4, m).astype(np.uint8)                 # mostly absent pieces
        else:
            o = int(rng.integers(0, g.size - m))
            r = g[o:o + m].copy()
            flip = rng.choice(m, size=min(m, int(rng.integers(0, 5))), replace=False)
            r[flip] = (r[flip] + rng.integers(1, 4, size=flip.size)) & 3
        reads.append(r)
        ks.append(int(rng.integers(0, 4)))
    return reads, ks


def test_lower_bound_words_equal_the_definition():
    g = gc.genome("1m").codes[:40_000]
    rng = np.random.default_rng(21)
    reads, ks = _reads_from(g, rng, 300)
    b = gc.batch_from_reads(reads, ks)
    idx = gc.mica().Index.build(synth.to_acgt_bytes(g), kmer_q=10, sa_sample=8)
    got = idx.debug_lower_bounds(b)
    for i, (r, k) in enumerate(zip(reads, ks)):
        for s, p in ((0, r), (1, refcheck.rc(r))):
            want = refcheck.lb_word(refcheck.lower_bound_breakpoints(g, p, k, 10))
            assert int(got[2 * i + s]) == want, (i, s, len(r), k)
    idx.free()


@pytest.mark.parametrize("kernel", KERNELS)
def test_pruned_equals_unpruned_equals_oracle(kernel):
    g = gc.genome("64m")
    b = synth.reads_uneven(g, n=200_000).subset(np.arange(0, 200_000, 100))   # 2,000 reads, k 0..3
    want = gc.oracle_index("64m").align(b, cap=1000)
    idx = gc.gpu_index("64m")
    got = idx.align_batch(b, hit_cap=1000, kernel=kernel, prune=True)
    pruned = idx.stats()
    gc.assert_same(got, want, "pruned")
    got = idx.align_batch(b, hit_cap=1000, kernel=kernel, prune=False)
    full = idx.stats()
    gc.assert_same(got, want, "unpruned")
    assert pruned["lb_steps"] > 0 and full["lb_steps"] == 0
    assert pruned["lb_dead_tasks"] > 0
    assert pruned["nodes"] < full["nodes"] and pruned["seeds"] < full["seeds"]


def test_index_with_and_without_lower_bounds(tmp_path):
    m = gc.mica()
    g = gc.genome("1m").codes[:60_000]
    rng = np.random.default_rng(22)
    reads, ks = _reads_from(g, rng, 200)
    b = gc.batch_from_reads(reads, ks)
    want = oracle.FMIndex(g, "sort").align(b, cap=1000)
    plain = m.Index.build(synth.to_acgt_bytes(g), kmer_q=10, sa_sample=8, lower_bounds=False)
    lbi = m.Index.build(synth.to_acgt_bytes(g), kmer_q=10, sa_sample=8, lower_bounds=True)
    assert plain.info()["lower_bounds"] == 0 and plain.info()["rev_occ_bytes"] == 0
    assert lbi.info()["lower_bounds"] == 1 and lbi.info()["rev_occ_bytes"] == lbi.info()["occ_bytes"]
    for idx in (plain, lbi):
        for kernel in KERNELS:
            gc.assert_same(idx.align_batch(b, hit_cap=1000, kernel=kernel), want, kernel)
    with pytest.raises(m.MicaError) as e:
        plain.debug_lower_bounds(b)
    assert e.value.code == m.MICA_EINVAL
    # the bidirectional search needs the reversed genome's index and q-mer table
    assert lbi.info()["rev_table_bytes"] == lbi.info()["table_bytes"] and plain.info()["rev_table_bytes"] == 0
    gc.assert_same(lbi.align_batch(b, hit_cap=1000, kernel="bidirectional"), want, "bidirectional")
    # without them the persistent kernel runs instead
    gc.assert_same(plain.align_batch(b, hit_cap=1000, kernel="bidirectional"), want, "bidirectional, no reversal")
    # the index file keeps (or omits) the reversed genome's blocks
    for idx, name in ((plain, "plain.mica"), (lbi, "lb.mica")):
        path = str(tmp_path / name)
        idx.save(path)
        back = m.Index.load(path)
        assert back.info() == idx.info()
        gc.assert_same(back.align_batch(b, hit_cap=1000), want, name)
        if idx is lbi:
            assert np.array_equal(back.debug_lower_bounds(b), lbi.debug_lower_bounds(b))
            gc.assert_same(back.align_batch(b, hit_cap=1000, kernel="bidirectional"), want, "loaded, bidirectional")
        back.free()
    plain.free()
    lbi.free()
