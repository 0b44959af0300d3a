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


def _decode_text(words, n):
    return ((words[:, None] >> (2 * np.arange(16, dtype=np.uint32))) & 3).astype(np.uint8).ravel()[:n]


def _check_full_sa(idx, g, sa):
    n = g.size
    got_sa = idx.debug_full_sa("sa")
    assert np.array_equal(got_sa, sa)
    isa = idx.debug_full_sa("isa")
    assert np.array_equal(isa[sa.astype(np.int64)], np.arange(n + 1, dtype=np.uint32))
    words = idx.debug_full_sa("text")
    assert words.size % 4 == 0 and words.size * 16 >= n + 64          # zero padding past the end
    assert np.array_equal(_decode_text(words, n), g)
    tail = _decode_text(words, words.size * 16)[n:]
    assert not tail.any()


@pytest.mark.parametrize("sa_sample", [1, 5, 16, 32])
@pytest.mark.parametrize("n", [1, 15, 16, 17, 33, 3001, 40_000])
def test_full_sa_built_and_rebuilt_at_load(tmp_path, sa_sample, n):
    """The whole suffix array, its inverse and the 2-bit text: at build time
    from the index's own suffix array, after a save and load by LF steps from
    the sampled rows (a walk from row 0 covers the positions above the last
    multiple of s); both equal the definitions."""
    rng = np.random.default_rng(n * 7 + sa_sample)
    g = (rng.integers(0, 4, n) if n % 2 else np.resize(rng.integers(0, 4, 5), n)).astype(np.uint8)
    m = gc.mica()
    sa = oracle.sa_sort(g)
    idx = m.Index.build(synth.to_acgt_bytes(g), kmer_q=min(8, max(1, n)), sa_sample=sa_sample)
    info = idx.info()
    assert info["full_sa"] == 1 and info["full_sa_bytes"] == 8 * (n + 1) + 4 * (((n + 15) // 16 + 7) // 4 * 4)
    _check_full_sa(idx, g, sa)
    path = str(tmp_path / "idx.mica")
    idx.save(path)
    idx2 = m.Index.load(path)
    assert idx2.info() == info
    _check_full_sa(idx2, g, sa)
    rows = np.arange(n + 1, dtype=np.uint64)
    assert np.array_equal(idx2.debug_locate(rows), sa)          # the LF walk still answers too
    idx.free(); idx2.free()


def test_full_sa_64m_and_without(tmp_path):
    """At 64 Mbp: the built arrays against the oracle's suffix array, and the
    arrays rebuilt from a saved file equal the built ones; an index built
    without them reports none and refuses the debug copy."""
    m = gc.mica()
    g = gc.genome("64m").codes
    idx = gc.gpu_index("64m")
    _check_full_sa(idx, g, gc.oracle_index("64m").sa())
    path = str(tmp_path / "idx64.mica")
    idx.save(path)
    idx2 = m.Index.load(path)
    for which in ("sa", "isa", "text"):
        assert np.array_equal(idx2.debug_full_sa(which), idx.debug_full_sa(which)), which
    idx2.free()
    small = g[:100_000]
    idx3 = m.Index.build(synth.to_acgt_bytes(small), kmer_q=10, sa_sample=16, full_sa=False)
    assert idx3.info()["full_sa"] == 0 and idx3.info()["full_sa_bytes"] == 0
    with pytest.raises(m.MicaError) as e:
        idx3.debug_full_sa("sa", 0, 10)
    assert e.value.code == m.MICA_EINVAL
    path3 = str(tmp_path / "idx_nofull.mica")
    idx3.save(path3)
    assert m.Index.load(path3).info()["full_sa"] == 0
    idx3.free()


def test_longer_seed_tables_are_sa_intervals(tmp_path):
    """The longer seed tables (q = ceil(log4(N + 1)) + 1 = 13 for 5 Mbp) of
    G$ and of G~$, built from the text at build time and again at load: every
    length <= 13, including the codes of the genome's last bases (short
    suffixes), gives the exact interval of backward search in the genome's
    and the reversed genome's index; the q-mer tables answer the same."""
    g = synth.repeat_genome(5_000_000, 7, copy_frac=0.1, copy_len=(500, 5000), tandem_frac=0.02).codes
    m = gc.mica()
    idx = m.Index.build(synth.to_acgt_bytes(g), kmer_q=12, sa_sample=16)
    info = idx.info()
    assert info["long_q"] == 13 and info["long_table_bytes"] == 2 * ((4 ** 13) + 1) * 4
    fm, rfm = oracle.FMIndex(g, "sais"), oracle.FMIndex(g[::-1].copy(), "sais")
    path = str(tmp_path / "idx5m.mica")
    idx.save(path)
    idx2 = m.Index.load(path)
    assert idx2.info() == info
    rng = np.random.default_rng(13)
    for length in (1, 6, 12, 13):
        ncode = 4 ** length
        tail = [int("".join(str(int(c)) for c in g[len(g) - j:][:length]).ljust(length, "0"), 4)
                for j in range(1, length + 1)]
        # G~'s last bases are G's first ones reversed: its short suffixes, padded
        head = [int("".join(str(int(c)) for c in g[:j][::-1]).ljust(length, "0"), 4) for j in range(1, length + 1)]
        planted = [int("".join(str(int(c)) for c in g[p0:p0 + length]), 4)
                   for p0 in rng.integers(0, len(g) - length, 300)]
        codes = np.unique(np.concatenate([rng.integers(0, ncode, 300), [0, ncode - 1], tail, head,
                                          planted])).astype(np.uint32)
        pats = [np.array([(int(x) >> (2 * (length - 1 - t))) & 3 for t in range(length)], np.uint8) for x in codes]
        want_f = [fm.exact_interval(p) for p in pats]
        want_r = [rfm.exact_interval(p) for p in pats]
        for which, want in (("long_fwd", want_f), ("long_rev", want_r)) + \
                (((("fwd", want_f), ("rev", want_r))) if length <= 12 else ()):
            for ix in (idx, idx2):
                got = ix.debug_table_interval(which, codes, length)
                for (l, r), (el, er) in zip(got, want):
                    assert (r - l) == (er - el), (which, length)
                    if el < er:
                        assert (int(l), int(r)) == (el, er), (which, length)
    with pytest.raises(m.MicaError):
        idx.debug_table_interval("long_fwd", np.zeros(1, np.uint32), 14)
    small = m.Index.build(synth.to_acgt_bytes(g[:100_000]), kmer_q=12, sa_sample=16)
    assert small.info()["long_q"] == 0                         # log4 N + 1 <= 12: no longer tables
    with pytest.raises(m.MicaError):
        small.debug_table_interval("long_fwd", np.zeros(1, np.uint32), 1)
    idx.free(); idx2.free(); small.free()


def test_gather_ceiling_orders_l2_above_hbm():
    """The random-gather ceiling: a buffer that fits L2 serves 32-byte random
    loads faster than one twelve times L2's size, and both stay below a
    plausible bound for one GB300 (L2 random reads well under 100 TB/s)."""
    m = gc.mica()
    l2 = m.gather_ceiling(64 << 20, 32, loads=1 << 26)
    hbm = m.gather_ceiling(3 << 29, 32, loads=1 << 26)
    assert 0 < hbm["gbs"] < l2["gbs"] < 100_000
    assert hbm["gbs"] < 10_000
