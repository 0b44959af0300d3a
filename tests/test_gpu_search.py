"""GPU k-mismatch search against the oracle, both kernels, bit-exact:
totals, CSR offsets and every (position, strand, mismatches)."""
import numpy as np
import pytest

import oracle
import synth
from tests import golden_cases, refcheck
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu
KERNELS = ["persistent", "plain", "plain_by_length", "bidirectional"]


@pytest.mark.parametrize("kernel", KERNELS)
def test_handworked(kernel):
    m = gc.mica()
    for case in golden_cases.cases():
        g = golden_cases.codes(case["genome"])
        idx = m.Index.build(case["genome"].encode(), kmer_q=2, sa_sample=2)
        b = golden_cases.batch_of(case["read"], case["k"])
        res = idx.align_batch(b, hit_cap=case["cap"], kernel=kernel)
        assert int(res.total[0]) == case["total"], case
        assert res.hits_of(0) == case["hits"], case
        idx.free()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("q", [5, 10, 12])
def test_slice_against_bruteforce(kernel, q):
    g, b = synth.slice_10k(gc.genome("1m"))
    idx = gc.mica().Index.build(synth.to_acgt_bytes(g.codes), kmer_q=q, sa_sample=8)
    for k in range(4):
        b.k[:] = k
        bf = oracle.bruteforce(g.codes, b)
        got = idx.align_batch(b, hit_cap=0, kernel=kernel)
        gc.assert_same(got, bf, f"k={k}")


@pytest.mark.parametrize("kernel", KERNELS)
def test_random_1m_10k_reads(kernel):
    g = gc.genome("1m")
    b = synth.reads_1m(g)
    want = gc.oracle_index("1m").align(b, cap=0)
    got = gc.gpu_index("1m").align_batch(b, hit_cap=0, kernel=kernel)
    gc.assert_same(got, want)
    # the closed form: every read hits exactly its origin
    assert np.array_equal(got.total, np.ones(b.n, np.uint64))
    assert np.array_equal(got.hits["pos"], b.origin.astype(np.uint32))


def _edge_batch(g, rng):
    n = g.size
    reads, ks = [], []
    for m in [1, 2, 3, 11, 12, 13, 15, 16, 17, 31, 32, 33, 63, 64, 65, 100, 150, 250, 255, 256]:
        for k in range(4):
            p = int(rng.integers(0, n - m + 1))
            r = g[p:p + m].copy()
            if rng.random() < 0.5:
                r = refcheck.rc(r)
            for q in rng.choice(m, size=min(m, k), replace=False):
                r[q] = (r[q] + rng.integers(1, 4)) & 3
            reads.append(r)
            ks.append(k)
    # palindromes (read == its reverse complement)
    for half in (2, 5, 8):
        h = rng.integers(0, 4, half).astype(np.uint8)
        reads.append(np.concatenate([h, refcheck.rc(h)]))
        ks.append(1)
    return gc.batch_from_reads(reads, ks)


@pytest.mark.parametrize("kernel", KERNELS)
def test_edge_lengths_and_budgets(kernel):
    rng = np.random.default_rng(21)
    g = synth.repeat_genome(30_000, 3, copy_frac=0.2, copy_len=(300, 2000), tandem_frac=0.1,
                            array_len=(100, 1500)).codes
    b = _edge_batch(g, rng)
    fm = oracle.FMIndex(g)
    for q, cap in ((12, 0), (8, 3), (4, 40)):
        idx = gc.mica().Index.build(synth.to_acgt_bytes(g), kmer_q=q, sa_sample=4)
        got = idx.align_batch(b, hit_cap=cap, kernel=kernel)
        gc.assert_same(got, fm.align(b, cap=cap), f"q={q} cap={cap}")
        idx.free()


@pytest.mark.parametrize("kernel", KERNELS)
def test_whole_genome_read(kernel):
    g = np.random.default_rng(4).integers(0, 4, 256).astype(np.uint8)
    reads = [g.copy(), refcheck.rc(g)]
    b = gc.batch_from_reads(reads, [3, 0])
    idx = gc.mica().Index.build(synth.to_acgt_bytes(g), kmer_q=12, sa_sample=16)
    got = idx.align_batch(b, hit_cap=0, kernel=kernel)
    gc.assert_same(got, oracle.FMIndex(g).align(b))


@pytest.mark.parametrize("kernel", KERNELS)
def test_many_hits_sort_paths(kernel):
    """Reads in tandem arrays: more than 32 hits (block sort) and, uncapped,
    more than 4096 hits (global sort)."""
    g = np.resize(np.array([0, 3, 3], np.uint8), 30_000)       # (ATT)^n
    g[::997] = 2
    fm = oracle.FMIndex(g)
    reads = [g[100:130].copy(), g[5:25].copy(), refcheck.rc(g[40:70])]
    b = gc.batch_from_reads(reads, [0, 1, 2])
    idx = gc.mica().Index.build(synth.to_acgt_bytes(g), kmer_q=12, sa_sample=16)
    for cap in (0, 100, 1000, 5000):
        got = idx.align_batch(b, hit_cap=cap, kernel=kernel)
        gc.assert_same(got, fm.align(b, cap=cap), f"cap={cap}")
    assert int(got.total.max()) > 4096


@pytest.mark.parametrize("kernel", KERNELS)
def test_many_intervals_and_the_cap(kernel):
    """Reads in a diverged (AC)^n array (4% substitutions) match thousands
    of distinct substrings within k: per read 4 to 6,588 SA intervals and
    4 to 18,580 hits.  Caps 1..5000 take every selection case: a short
    interval list over the cap, a long one over the cap (threshold found
    without sorting), a long one within the cap, and uncapped lists above
    the shared-memory sort size."""
    rng = np.random.default_rng(7)
    core = np.resize(np.array([0, 1], np.uint8), 40_000)
    mut = rng.random(core.size) < 0.04
    core[mut] = (core[mut] + rng.integers(1, 4, size=int(mut.sum()))) & 3
    g = np.concatenate([rng.integers(0, 4, 20_000).astype(np.uint8), core,
                        rng.integers(0, 4, 20_000).astype(np.uint8)])
    m = 40
    reads = [g[20_000 + i * 1_999: 20_000 + i * 1_999 + m].copy() for i in range(20)]
    reads += [refcheck.rc(r) for r in reads[:5]]
    b = gc.batch_from_reads(reads, [2] * 20 + [3] * 5)
    fm = oracle.FMIndex(g)
    idx = gc.mica().Index.build(synth.to_acgt_bytes(g), kmer_q=10, sa_sample=8)
    for cap in (0, 1, 7, 100, 1000, 5000):
        got = idx.align_batch(b, hit_cap=cap, kernel=kernel)
        gc.assert_same(got, fm.align(b, cap=cap), f"cap={cap}")
    assert int(got.total.max()) > 18_000
    idx.free()


def test_graph_path_interval_overflow_falls_back():
    """A captured batch whose search overflows the interval buffer (64 reads
    with thousands of leaf intervals each, far above the 4 per read plus
    65,536 it is sized for) leaves the post kernels idle and falls back to
    the regular path, which grows the buffer: the result is the oracle's."""
    rng = np.random.default_rng(8)
    core = np.resize(np.array([0, 1], np.uint8), 40_000)
    mut = rng.random(core.size) < 0.04
    core[mut] = (core[mut] + rng.integers(1, 4, size=int(mut.sum()))) & 3
    g = np.concatenate([rng.integers(0, 4, 10_000).astype(np.uint8), core])
    reads = [g[10_000 + i * 600: 10_000 + i * 600 + 40].copy() for i in range(64)]
    b = gc.batch_from_reads(reads, [3] * 64)
    idx = gc.mica().Index.build(synth.to_acgt_bytes(g), kmer_q=10, sa_sample=8)
    want = oracle.FMIndex(g).align(b, cap=1000)
    for call in range(2):
        got = idx.align_batch(b, hit_cap=1000, kernel="persistent")
        st = idx.stats()
        gc.assert_same(got, want, f"call {call}")
        assert st["intervals"] > 4 * 64 + 65_536
    idx.free()


@pytest.mark.parametrize("kernel", KERNELS)
def test_empty_batch(kernel):
    idx = gc.gpu_index("1m")
    b = gc.batch_from_reads([], [])
    res = idx.align(np.zeros(0, np.uint32), np.zeros(1, np.uint64), np.zeros(0, np.uint16),
                    np.zeros(0, np.uint8), kernel=kernel)
    assert res.total.size == 0 and res.hits.size == 0 and list(res.offsets) == [0]


def test_rejects_invalid_reads():
    m = gc.mica()
    idx = gc.gpu_index("1m")
    for m_len, k in ((0, 0), (257, 0), (10, 4)):
        words = np.zeros(32, np.uint32)
        off = np.array([0, 17], np.uint64)
        with pytest.raises(m.MicaError) as e:
            idx.align(words, off, np.array([m_len], np.uint16), np.array([k], np.uint8))
        assert e.value.code == m.MICA_EINVAL
    # word offsets pointing past the packed words
    with pytest.raises(m.MicaError):
        idx.align(np.zeros(2, np.uint32), np.array([0, 2], np.uint64), np.array([100], np.uint16),
                  np.array([1], np.uint8))


@pytest.mark.parametrize("kernel", KERNELS)
def test_repeats_64m_sample(kernel):
    g = gc.genome("64m")
    b = synth.reads_64m(g, n=1_000_000).subset(np.arange(0, 1_000_000, 250))   # 4,000 reads
    want = gc.oracle_index("64m").align(b, cap=1000)
    got = gc.gpu_index("64m").align_batch(b, hit_cap=1000, kernel=kernel)
    gc.assert_same(got, want)


@pytest.mark.parametrize("kernel", KERNELS)
def test_uneven_64m_sample(kernel):
    g = gc.genome("64m")
    full = synth.reads_uneven(g, n=200_000)
    b = full.subset(np.arange(0, full.n, 100))                                     # 2,000 reads
    want = gc.oracle_index("64m").align(b, cap=1000)
    got = gc.gpu_index("64m").align_batch(b, hit_cap=1000, kernel=kernel)
    gc.assert_same(got, want)


def test_uneven_64m_100k_reads_equal_oracle():
    """100,000 reads of the benchmark's uneven 1M-read batch (every tenth:
    lengths 50-250, k 0..3, 30% from repeats) equal the oracle for the
    persistent kernel and the per-length plain launches."""
    g = gc.genome("64m")
    b = synth.reads_uneven(g, n=1_000_000).subset(np.arange(0, 1_000_000, 10))
    want = gc.oracle_index("64m").align(b, cap=1000)
    idx = gc.gpu_index("64m")
    for kernel in ("persistent", "plain_by_length", "bidirectional"):
        gc.assert_same(idx.align_batch(b, hit_cap=1000, kernel=kernel), want, kernel)
    assert int(want.total.max()) > 1000 and np.count_nonzero(b.k == 3) > 20_000


def test_pipelined_submit_and_collect():
    """Pipelined host batches: two slots in flight, results equal to the
    one-call path and the oracle, collected in either order; a third submit
    is refused (MICA_EBUSY) and a collected ticket is unknown (MICA_ENOTFOUND);
    a bad batch is refused at submit without taking a slot; the persistent
    and plain kernels and best-stratum reporting go through the same slots."""
    m = gc.mica()
    g = gc.genome("64m")
    fm = gc.oracle_index("64m")
    idx = gc.gpu_index("64m")
    u = synth.reads_uneven(g, n=200_000)
    parts = [u.subset(np.arange(i, 200_000, 400)) for i in range(4)]          # 4 x 500 reads
    want = [fm.align(b, cap=1000) for b in parts]
    t0 = idx.submit_batch(parts[0])
    t1 = idx.submit_batch(parts[1])
    with pytest.raises(m.MicaError) as e:
        idx.submit_batch(parts[2])
    assert e.value.code == m.MICA_EBUSY
    gc.assert_same(idx.collect(t1), want[1], "second collected first")
    t2 = idx.submit_batch(parts[2])
    gc.assert_same(idx.collect(t0), want[0], "first")
    with pytest.raises(m.MicaError) as e:
        idx.collect(t0)
    assert e.value.code == m.MICA_ENOTFOUND
    bad = parts[3]
    with pytest.raises(m.MicaError) as e:
        idx.submit(bad.words, bad.word_off, np.full(bad.n, 300, np.uint16), bad.k)
    assert e.value.code == m.MICA_EINVAL
    t3 = idx.submit_batch(parts[3])
    gc.assert_same(idx.collect(t2), want[2], "third")
    gc.assert_same(idx.collect(t3), want[3], "fourth")
    # a steady stream, as the benchmark runs it: submit the next, collect the previous
    prev = None
    for r in range(6):
        t = idx.submit_batch(parts[r % 4], kernel=("bidirectional", "persistent", "plain")[r % 3])
        if prev is not None:
            gc.assert_same(idx.collect(prev[0]), want[prev[1]], f"stream {r}")
        prev = (t, r % 4)
    gc.assert_same(idx.collect(prev[0]), want[prev[1]], "stream end")
    tb = idx.submit_batch(parts[0], kernel="persistent", report="best_stratum")
    gc.assert_same(idx.collect(tb), fm.align_best_stratum(parts[0], cap=1000), "best stratum")
    assert idx.stats()["tasks"] == 2 * parts[0].n


def test_free_with_batches_in_flight():
    """An index freed with two submitted batches never collected waits for
    them (nothing they read is released under them) and leaves the device
    usable: a new index of the same genome gives the oracle's result."""
    m = gc.mica()
    g = gc.genome("1m")
    b = synth.reads_1m(g, n=2_000)
    idx = m.Index.build(synth.to_acgt_bytes(g.codes), kmer_q=10, sa_sample=8)
    idx.submit_batch(b)
    idx.submit_batch(b, kernel="persistent")
    idx.free()
    idx2 = m.Index.build(synth.to_acgt_bytes(g.codes), kmer_q=10, sa_sample=8)
    try:
        gc.assert_same(idx2.align_batch(b, hit_cap=1000), gc.oracle_index("1m").align(b, cap=1000), "after free")
    finally:
        idx2.free()


def test_bidirectional_text_check_settings():
    """One-row intervals checked against the text (the whole suffix array,
    its inverse and the 2-bit text resident): with the check after 1, 24 or the
    default 12 matched bases (24: the one-row node first takes base-by-base
    steps past the 12-base seed), with it off (256), and on an index without the
    arrays, every result equals the oracle, on the uneven 64 Mbp sample
    (k 0..3, lengths 50..250, reads inside planted repeats) and on diverged
    (AC)^n reads, with and without a cap and with small node budgets."""
    g = gc.genome("64m")
    b = synth.reads_uneven(g, n=200_000).subset(np.arange(0, 200_000, 100))   # 2,000 reads
    want = gc.oracle_index("64m").align(b, cap=1000)
    idx = gc.gpu_index("64m")
    try:
        for verify in (1, 24, 0, 256):
            for budget in (0, 16):
                idx.set_tuning(bidir_verify=verify, bidir_budget=budget)
                got = idx.align_batch(b, hit_cap=1000, kernel="bidirectional")
                gc.assert_same(got, want, f"verify {verify} budget {budget}")
                st = idx.stats()
                assert (st["verified"] > 0) == (verify < 256), (verify, st["verified"])
                assert (st["verify_bytes"] > 0) == (verify < 256)
        # both compiled shapes (64 task slots per warp, 6 warps; 32 slots, 8 warps)
        for shape in (0, 1):
            for budget in (0, 16):
                idx.set_tuning(bidir_shape=shape, bidir_budget=budget)
                gc.assert_same(idx.align_batch(b, hit_cap=1000, kernel="bidirectional"), want,
                               f"shape {shape} budget {budget}")
        with pytest.raises(gc.mica().MicaError):
            idx.set_tuning(bidir_shape=2)
    finally:
        idx.set_tuning()
    rng = np.random.default_rng(9)
    core = np.resize(np.array([0, 1], np.uint8), 30_000)
    mut = rng.random(core.size) < 0.04
    core[mut] = (core[mut] + rng.integers(1, 4, size=int(mut.sum()))) & 3
    tg = np.concatenate([rng.integers(0, 4, 20_000).astype(np.uint8), core, rng.integers(0, 4, 5_000).astype(np.uint8)])
    reads = [tg[i: i + 60].copy() for i in range(0, 55_000 - 60, 2_300)]
    tb = gc.batch_from_reads(reads, [2] * (len(reads) // 2) + [3] * (len(reads) - len(reads) // 2))
    tfm = oracle.FMIndex(tg)
    m = gc.mica()
    for full_sa in (True, False):
        tidx = m.Index.build(synth.to_acgt_bytes(tg), kmer_q=10, sa_sample=8, full_sa=full_sa)
        for verify in (1, 0):
            tidx.set_tuning(bidir_verify=verify)
            for cap in (0, 7):
                got = tidx.align_batch(tb, hit_cap=cap, kernel="bidirectional")
                gc.assert_same(got, tfm.align(tb, cap=cap), f"tandem full_sa={full_sa} verify {verify} cap={cap}")
                assert (tidx.stats()["verified"] > 0) == full_sa
        tidx.free()


def test_bidirectional_odd_batch_above_half_million():
    """A batch of an odd number of reads above 2^19: each frontier buffer then
    holds 2n items, and the second one must still start on a 16-byte
    boundary for the kernel's 16-byte item loads and stores.  Budgets of 2 and
    8 nodes send many nodes through several rounds, which alternate between
    the two buffers; the result equals the persistent kernel's."""
    g = gc.genome("64m")
    b = synth.reads_64m(g, n=600_001)
    assert b.n % 2 == 1 and b.n > 1 << 19
    idx = gc.gpu_index("64m")
    want = idx.align_batch(b, hit_cap=1000, kernel="persistent")
    try:
        for budget in (2, 8, 0):
            idx.set_tuning(bidir_budget=budget)
            got = idx.align_batch(b, hit_cap=1000, kernel="bidirectional")
            gc.assert_same(got, want, f"budget {budget}")
            if budget:
                assert idx.stats()["spills"] > 50_000       # many nodes went through later rounds
    finally:
        idx.set_tuning()


def test_bidirectional_frontier_rounds_and_give_up():
    """The bidirectional kernel's budget: a task over its node budget exports
    its pending nodes, and further launches continue them as tasks of their
    own; a read still exporting after the last round is given up, its leaves
    dropped and the read searched again by the persistent kernel.  Budgets of
    200 and 8 nodes take many reads through the rounds, a budget of 1 through
    the give-up path (walks of 100+ steps need more than 64 rounds), on the
    uneven 64 Mbp sample (k 0..3) and on diverged (AC)^n reads with thousands
    of leaves; every result equals the oracle, on repeated calls (the
    captured-graph path steps aside once a batch needed more)."""
    g = gc.genome("64m")
    b = synth.reads_uneven(g, n=200_000).subset(np.arange(0, 200_000, 100))   # 2,000 reads
    want = gc.oracle_index("64m").align(b, cap=1000)
    idx = gc.gpu_index("64m")
    try:
        for budget in (200, 8, 1):
            idx.set_tuning(bidir_budget=budget)
            for call in range(2):
                got = idx.align_batch(b, hit_cap=1000, kernel="bidirectional")
                gc.assert_same(got, want, f"budget {budget}, call {call}")
                st = idx.stats()
                assert st["spills"] > 0                                # nodes exported to later rounds
                if budget == 1:
                    assert st["fallback_reads"] > 0                    # and reads given up
        idx.set_tuning()
        gc.assert_same(idx.align_batch(b, hit_cap=1000, kernel="bidirectional"), want, "default budget")
    finally:
        idx.set_tuning()
    rng = np.random.default_rng(7)
    core = np.resize(np.array([0, 1], np.uint8), 40_000)
    mut = rng.random(core.size) < 0.04
    core[mut] = (core[mut] + rng.integers(1, 4, size=int(mut.sum()))) & 3
    tg = np.concatenate([rng.integers(0, 4, 20_000).astype(np.uint8), core])
    reads = [tg[20_000 + i * 1_999: 20_000 + i * 1_999 + 40].copy() for i in range(16)]
    tb = gc.batch_from_reads(reads, [2] * 8 + [3] * 8)
    tfm = oracle.FMIndex(tg)
    tidx = gc.mica().Index.build(synth.to_acgt_bytes(tg), kmer_q=10, sa_sample=8)
    for budget in (200, 1):
        tidx.set_tuning(bidir_budget=budget)
        for cap in (0, 1000):
            got = tidx.align_batch(tb, hit_cap=cap, kernel="bidirectional")
            gc.assert_same(got, tfm.align(tb, cap=cap), f"tandem budget {budget} cap={cap}")
            assert tidx.stats()["spills"] > 0
    tidx.free()


def test_every_shape_and_block_gives_the_same_result():
    g = gc.genome("64m")
    full = synth.reads_uneven(g, n=200_000)
    b = full.subset(np.arange(0, full.n, 40))                                      # 5,000 reads
    idx = gc.gpu_index("64m")
    ref = idx.align_batch(b, hit_cap=1000, kernel="plain")
    m = gc.mica()
    try:
        for shape in range(len(m.tuning_shapes())):
            idx.set_tuning(shape=shape)
            gc.assert_same(idx.align_batch(b, hit_cap=1000, kernel="persistent"), ref, f"shape {shape}")
        idx.set_tuning(plain_block=64, plain_budget=100, plain_block_len=(32, 96, 256, 512))
        for kernel in ("plain", "plain_by_length"):
            got = idx.align_batch(b, hit_cap=1000, kernel=kernel)
            gc.assert_same(got, ref, f"{kernel} with a 100-node budget")
            assert idx.stats()["spills"] > 0          # the re-queue path ran
        with pytest.raises(m.MicaError):
            idx.set_tuning(shape=99)
    finally:
        idx.set_tuning()


def test_full_1m_reads_64m():
    """Full 1M x 150 bp batch on the 64 Mbp repeat genome in the launch shape
    the benchmark times: every read's total, offsets and hits equal the
    oracle's for both kernels; every hit's mismatch count is recomputed from
    the genome on a sample."""
    g = gc.genome("64m")
    b = synth.reads_64m(g)
    idx = gc.gpu_index("64m")
    want = gc.oracle_index("64m").align(b, cap=1000)
    a = idx.align_batch(b, hit_cap=1000, kernel="persistent")
    gc.assert_same(a, want, "persistent vs oracle, 1M reads")
    p = idx.align_batch(b, hit_cap=1000, kernel="plain")
    gc.assert_same(p, want, "plain vs oracle, 1M reads")
    gc.assert_same(idx.align_batch(b, hit_cap=1000, kernel="bidirectional"), want, "bidirectional vs oracle, 1M reads")
    rng = np.random.default_rng(99)
    # invariants on every read
    cnt = np.diff(a.offsets.astype(np.int64))
    assert np.all(cnt == np.minimum(a.total.astype(np.int64), 1000))
    assert np.all(a.hits["mm"] <= 2)
    assert np.all(a.hits["pos"].astype(np.int64) <= g.n - 150)
    for i in rng.choice(b.n, 300, replace=False):
        r = b.read(int(i))
        for pos, s, d in a.hits_of(int(i)):
            w = g.codes[pos:pos + 150]
            assert int(((refcheck.rc(r) if s else r) != w).sum()) == d


def test_autotune_cache_and_results_unchanged(tmp_path):
    g = gc.genome("64m")
    full = synth.reads_uneven(g, n=200_000)
    b = full.subset(np.arange(0, full.n, 50))                                      # 4,000 reads
    idx = gc.gpu_index("64m")
    m = gc.mica()
    cache = str(tmp_path / "tuning.txt")
    try:
        ref = idx.align_batch(b, hit_cap=1000, kernel="plain")
        t = idx.autotune(b, repeats=1, cache=cache)
        assert 0 <= t["shape"] < len(m.tuning_shapes())
        assert t["plain_block"] in (64, 128, 256, 512)
        assert all(x in (64, 128, 256, 512) for x in t["plain_block_len"])    # all four classes present
        assert t["bidir_shape"] in (0, 1) and t["bidir_budget"] in (1024, 4096)
        idx.set_tuning()
        assert idx.autotune(b, cache=cache) == t                               # served from the cache
        for kernel in ("persistent", "plain", "plain_by_length", "bidirectional"):
            gc.assert_same(idx.align_batch(b, hit_cap=1000, kernel=kernel), ref, kernel)
    finally:
        idx.set_tuning()


def test_graph_replay_and_fallback():
    """Repeated batch shapes replay one captured CUDA graph with the same
    results; a batch whose hits overflow the graph's buffers falls back to
    the regular path and is still exact."""
    import torch
    m = gc.mica()
    g = gc.genome("64m")
    b = synth.reads_64m(g, n=20_000)
    idx = gc.gpu_index("64m")
    dev = torch.device("cuda", 0)
    d = (torch.from_numpy(b.words.view(np.int32)).to(dev), torch.from_numpy(b.word_off.view(np.int64)).to(dev),
         torch.from_numpy(b.lengths.view(np.int16)).to(dev), torch.from_numpy(b.k).to(dev))
    want = gc.oracle_index("64m").align(b, cap=1000)
    seen = []
    for call in range(3):
        r = idx.align_device(*d, b.n, hit_cap=1000)
        st = idx.stats()
        seen.append((st["graph_captures"], st["graph_replays"]))
        t, o, h = r.tensors()
        got = gc.mica().Result(t.cpu().numpy().view(np.uint64), o.cpu().numpy().view(np.uint64),
                               h.cpu().numpy().view(m.HIT_DTYPE))
        gc.assert_same(got, want, f"call {call}")
    assert seen[0] == (1, 1) and seen[1] == (0, 1) and seen[2] == (0, 1)
    # many hits per read: (AT)-rich genome, uncapped -> more hits than the graph's buffer holds
    tg = np.resize(np.array([0, 3], np.uint8), 200_000)
    tg[::1001] = 1
    tidx = m.Index.build(synth.to_acgt_bytes(tg), kmer_q=10, sa_sample=8)
    reads = gc.batch_from_reads([tg[10:40].copy() for _ in range(12)], [1] * 12)
    tw = (torch.from_numpy(reads.words.view(np.int32)).to(dev), torch.from_numpy(reads.word_off.view(np.int64)).to(dev),
          torch.from_numpy(reads.lengths.view(np.int16)).to(dev), torch.from_numpy(reads.k).to(dev))
    r = tidx.align_device(*tw, reads.n, hit_cap=0)
    assert tidx.stats()["graph_fallbacks"] == 1
    t, o, h = r.tensors()
    got = gc.mica().Result(t.cpu().numpy().view(np.uint64), o.cpu().numpy().view(np.uint64),
                           h.cpu().numpy().view(m.HIT_DTYPE))
    gc.assert_same(got, oracle.FMIndex(tg).align(reads, cap=0), "fallback")
    tidx.free()


@pytest.mark.parametrize("kernel", KERNELS)
def test_best_stratum_reporting(kernel):
    """MICA_REPORT_BEST_STRATUM = the oracle's best-stratum result: on the
    uneven 64 Mbp sample (k 0..3; caps 1000 and 3) and on the diverged
    (AC)^n fixture whose reads have thousands of intervals (caps 0, 1, 7)."""
    g = gc.genome("64m")
    b = synth.reads_uneven(g, n=200_000).subset(np.arange(0, 200_000, 200))     # 1,000 reads
    fm = gc.oracle_index("64m")
    idx = gc.gpu_index("64m")
    for cap in (1000, 3):
        got = idx.align_batch(b, hit_cap=cap, kernel=kernel, report="best_stratum")
        gc.assert_same(got, fm.align_best_stratum(b, cap=cap), f"64m cap={cap}")
    rng = np.random.default_rng(7)
    core = np.resize(np.array([0, 1], np.uint8), 40_000)
    mut = rng.random(core.size) < 0.04
    core[mut] = (core[mut] + rng.integers(1, 4, size=int(mut.sum()))) & 3
    tg = np.concatenate([rng.integers(0, 4, 20_000).astype(np.uint8), core])
    reads = [tg[20_000 + i * 1_999: 20_000 + i * 1_999 + 40].copy() for i in range(12)]
    tb = gc.batch_from_reads(reads, [2] * 8 + [3] * 4)
    tfm = oracle.FMIndex(tg)
    tidx = gc.mica().Index.build(synth.to_acgt_bytes(tg), kmer_q=10, sa_sample=8)
    for cap in (0, 1, 7):
        got = tidx.align_batch(tb, hit_cap=cap, kernel=kernel, report="best_stratum")
        gc.assert_same(got, tfm.align_best_stratum(tb, cap=cap), f"tandem cap={cap}")
    tidx.free()
