"""Human-scale parity: the 3.1 Gbp synthetic genome (about 45% repeats)
resident in HBM, paired 150 bp mates with k <= 2 and cap 1000, in the
launch shape the human-scale benchmark uses.

The oracle cannot build its index for 3.1 Gbp within a test, so sampled
reads are checked one by one against its brute-force Hamming scan of both
strands (exact totals; exact hit lists where the total is within the cap;
listed hits a subset otherwise), for the persistent and the bidirectional
kernel, every read against properties that hold at any size, and the
kernels against each other on every mate."""
import numpy as np
import pytest

import oracle
import synth
from tests import gpu_common as gc
from tests import refcheck

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def human():
    g = synth.human_genome()
    donor = synth.donor_of(g)
    b = synth.paired_reads(donor, 10_000)                       # 20,000 mates
    idx = gc.mica().Index.build(synth.to_acgt_bytes(g.codes), kmer_q=12, sa_sample=16)
    yield g, b, idx
    idx.free()


def test_human_sampled_reads_equal_bruteforce(human):
    g, b, idx = human
    rng = np.random.default_rng(44)
    sample = np.sort(rng.choice(b.n, 16, replace=False))
    sub = b.subset(sample)
    bf = oracle.bruteforce(g.codes, sub)
    for kernel in ("persistent", "bidirectional"):
        res = idx.align_batch(b, hit_cap=1000, kernel=kernel)
        for j, i in enumerate(sample):
            got = res.hits_of(int(i))
            want = bf.as_tuples(j)
            assert int(res.total[i]) == len(want), (kernel, int(i))
            if len(want) <= 1000:
                assert got == want, (kernel, int(i))
            else:
                assert len(got) == 1000 and set(got) <= set(want), (kernel, int(i))


def test_human_properties_and_kernels_agree(human):
    g, b, idx = human
    res = idx.align_batch(b, hit_cap=1000, kernel="persistent")
    cnt = np.diff(res.offsets.astype(np.int64))
    assert np.all(cnt == np.minimum(res.total.astype(np.int64), 1000))
    assert np.all(res.hits["mm"] <= 2)
    assert np.all(res.hits["pos"].astype(np.int64) <= g.n - 150)
    # most mates carry at most two differences from the reference
    assert np.mean(res.total > 0) > 0.7
    rng = np.random.default_rng(45)
    for i in rng.choice(b.n, 100, replace=False):
        r = b.read(int(i))
        hits = res.hits_of(int(i))
        key = [(p, s) for p, s, _ in hits]
        assert key == sorted(key)
        for p, s, d in hits[:20]:
            w = g.codes[p:p + 150]
            assert int(((refcheck.rc(r) if s else r) != w).sum()) == d
    sub = b.subset(np.arange(0, 4_000))
    gc.assert_same(idx.align_batch(sub, hit_cap=1000, kernel="plain"),
                   idx.align_batch(sub, hit_cap=1000, kernel="persistent"), "plain vs persistent")
    # the bidirectional kernel (text checks over the whole SA, rows past 2^31) on every mate
    gc.assert_same(idx.align_batch(b, hit_cap=1000, kernel="bidirectional"), res, "bidirectional vs persistent")


def test_human_serving_alone_equals_mix(human):
    """Serving on the resident 3.1 Gbp index (the serving workload's index):
    requests of mixed sizes, lengths and budgets submitted concurrently share
    ticks, and each result is bit-identical to the same request aligned
    alone; the alone results are pinned above (brute force and properties)."""
    import threading
    g, b, idx = human
    donor = synth.donor_of(g)
    reqs = synth.serve_requests(donor, 9, seed=47, size_range=(200, 6_000))
    alone = [idx.align_batch(r, hit_cap=1000) for r in reqs]
    ids = [None] * len(reqs)
    with gc.mica().Server(idx, hit_cap=1000, workers=2, max_tick_reads=8_000) as srv:
        def client(j0):
            for j in range(j0, len(reqs), 3):
                ids[j] = srv.submit_batch(reqs[j])
        th = [threading.Thread(target=client, args=(j,)) for j in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for j, rid in enumerate(ids):
            got, lat = srv.wait(rid)
            gc.assert_same(got, alone[j], f"request {j}")
        assert srv.stats()["ticks"] >= 1
    assert sum(int(r.offsets[-1]) for r in alone) > 0
