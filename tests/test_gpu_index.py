"""GPU index construction against the oracle: suffix array, occurrence
counts, q-mer table bounds and SA resolution by LF walks."""
import numpy as np
import pytest

import oracle
import synth
from tests import gpu_common as gc
from tests import refcheck

pytestmark = pytest.mark.gpu


def _strings():
    rng = np.random.default_rng(17)
    yield "empty", np.zeros(0, np.uint8)
    yield "one", np.array([2], np.uint8)
    yield "allA", np.zeros(5000, np.uint8)
    yield "AC", np.resize(np.array([0, 1], np.uint8), 4001)
    yield "period7", np.resize(rng.integers(0, 4, 7).astype(np.uint8), 30000)
    yield "random", rng.integers(0, 4, 100_000).astype(np.uint8)
    yield "repeats", synth.repeat_genome(200_000, 5, copy_frac=0.2, copy_len=(500, 5000), tandem_frac=0.1).codes


@pytest.mark.parametrize("name,g", list(_strings()), ids=[n for n, _ in _strings()])
def test_suffix_array_matches_oracle(name, g):
    got = gc.mica().debug_suffix_array(synth.to_acgt_bytes(g))
    want = oracle.sa_sort(g) if g.size <= 200_000 else oracle.sa_is(g)
    assert np.array_equal(got, want)


def test_suffix_array_64m_matches_sais():
    g = gc.genome("64m").codes
    got = gc.mica().debug_suffix_array(synth.to_acgt_bytes(g))
    assert np.array_equal(got, gc.oracle_index("64m").sa())


@pytest.mark.parametrize("name", ["1m", "64m"])
def test_occ_and_locate_match_oracle(name):
    fm = gc.oracle_index(name)
    idx = gc.gpu_index(name)
    rng = np.random.default_rng(3)
    rows = np.concatenate([rng.integers(0, fm.rows + 1, 20000),
                           np.arange(0, min(fm.rows, 192 * 4) + 1),
                           np.array([fm.rows - 1, fm.rows])]).astype(np.uint64)
    occ = idx.debug_occ(rows)
    want = np.array([[fm.occ(c, int(j)) for c in range(4)] for j in rows], dtype=np.uint32)
    assert np.array_equal(occ, want)
    sa = fm.sa()
    lrows = rng.integers(0, fm.rows, 20000).astype(np.uint64)
    assert np.array_equal(idx.debug_locate(lrows), sa[lrows.astype(np.int64)])
    info = idx.info()
    assert info["C"][:4] == [fm.C(c) for c in range(4)] and info["C"][4] == fm.rows


@pytest.mark.parametrize("sa_sample", [1, 5, 32])
def test_locate_every_row_small(sa_sample):
    g = np.random.default_rng(8).integers(0, 4, 3000).astype(np.uint8)
    idx = gc.mica().Index.build(synth.to_acgt_bytes(g), kmer_q=6, sa_sample=sa_sample)
    rows = np.arange(g.size + 1, dtype=np.uint64)
    assert np.array_equal(idx.debug_locate(rows), oracle.sa_sort(g))


@pytest.mark.parametrize("q", [1, 4, 8, 12])
def test_seed_intervals_are_sa_intervals(q):
    """Every length <= q: the table lookup equals exact backward search,
    including the codes next to the genome's last bases (short suffixes)."""
    g = synth.repeat_genome(20_000, 2, copy_frac=0.1, copy_len=(200, 1000), tandem_frac=0.05).codes
    idx = gc.mica().Index.build(synth.to_acgt_bytes(g), kmer_q=q, sa_sample=16)
    fm = oracle.FMIndex(g)
    rng = np.random.default_rng(q)
    for length in sorted({1, max(1, q // 2), q}):
        ncode = 4 ** length
        tail = [int("".join(str(int(c)) for c in g[len(g) - j:][:length]).ljust(length, "0"), 4)
                for j in range(1, length + 1)]
        near = [min(ncode - 1, c + d) for c in tail for d in (-1, 0, 1) if c + d >= 0]
        codes = np.unique(np.concatenate([rng.integers(0, ncode, 400), [0, ncode - 1], near])).astype(np.uint32)
        got = idx.debug_seed_interval(codes, length)
        for x, (l, r) in zip(codes, got):
            p = np.array([(int(x) >> (2 * (length - 1 - t))) & 3 for t in range(length)], np.uint8)
            el, er = fm.exact_interval(p)
            assert (r - l) == (er - el) == refcheck.count_occurrences(g, p)
            if el < er:
                assert (int(l), int(r)) == (el, er)


def test_save_load_roundtrip(tmp_path):
    g = gc.genome("1m").codes[:50_000]
    m = gc.mica()
    idx = m.Index.build(synth.to_acgt_bytes(g), kmer_q=10, sa_sample=8)
    path = str(tmp_path / "idx.mica")
    idx.save(path)
    idx2 = m.Index.load(path)
    assert idx.info() == idx2.info()
    rows = np.arange(0, g.size + 1, 7, dtype=np.uint64)
    assert np.array_equal(idx.debug_locate(rows), idx2.debug_locate(rows))
    assert np.array_equal(idx.debug_occ(rows), idx2.debug_occ(rows))


def test_gather_ceiling_orders_l2_above_hbm():
    """The random-gather ceiling: a buffer that fits L2 serves 32-byte random
    loads faster than one twelve times L2's size, and both stay below a
    plausible bound for one GB300 (L2 random reads well under 100 TB/s)."""
    m = gc.mica()
    l2 = m.gather_ceiling(64 << 20, 32, loads=1 << 26)
    hbm = m.gather_ceiling(3 << 29, 32, loads=1 << 26)
    assert 0 < hbm["gbs"] < l2["gbs"] < 100_000
    assert hbm["gbs"] < 10_000
