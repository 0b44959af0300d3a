"""SAM output (host-side, no GPU): the library's mica_sam_* writer against a
plain-Python restatement of the same rules (tests/samcheck.py), on oracle
results over a reference of several contigs with ambiguous bases, and
against what SAM itself fixes, checked on the records alone: SEQ, NM and MD
reproduce the contig's own bytes at POS, FLAG 16 iff SEQ is the reverse
complement of the read, one primary record per read, and mate fields that
point at each other."""

import os

import numpy as np
import pytest

import oracle
import synth
from tests import hostlib, samcheck

NAMES = ["chr1", "chr2", "chrUn_1", "chrM"]
WINDOW = (200, 600)


@pytest.fixture(scope="module")
def mica():
    return hostlib.mica()


@pytest.fixture(scope="module")
def setup(mica):
    contigs = synth.multi_contig_reference()
    g, starts, runs = oracle.reference_concat(contigs)
    ref = mica.Reference.create(b"".join(contigs), [len(c) for c in contigs], NAMES)
    return contigs, g, starts, runs, ref, oracle.FMIndex(g)


@pytest.fixture(scope="module")
def single(setup):
    contigs, g, starts, runs, ref, fm = setup
    rng = np.random.Generator(np.random.PCG64(synth.SEED_REFERENCE_READS + 1))
    regions = [(max(0, s - 120), min(len(g), s + 120), "boundary") for s in starts[1:-1]]
    regions += [(max(0, s - 120), min(len(g), e + 120), "ambiguous") for s, e in runs]
    regions += [(100, 500, "shared"), (starts[3] + 50, starts[3] + 450, "near copy")]
    n = 300
    lengths = rng.choice(np.array([60, 100]), size=n)
    k = rng.integers(0, 4, size=n, dtype=np.uint8)
    return synth.sample_reads(synth.Genome(g, regions), lengths, k, rng, subs="count", max_subs=3,
                              repeat_frac=0.6)


@pytest.fixture(scope="module")
def paired(setup):
    g = setup[1]
    return synth.paired_reads(g, 150, seed=synth.SEED_REFERENCE_READS + 2, m=100, insert_mean=350.0,
                              insert_sd=40.0)


def _write(mica, path, ref, batches, **kw):
    with mica.SamWriter(str(path), ref, **kw) as w:
        for batch, res, pairs in batches:
            w.write(batch, res, pairs)
    return open(path).read()


def _expected(setup, batch, res, pairs=None, **kw):
    contigs, g, starts, runs, ref, fm = setup
    return samcheck.sam_text(NAMES, starts, runs, synth.to_acgt_bytes(g).decode(), batch, res, pairs, **kw)


def _parse(text):
    return [line.split("\t") for line in text.splitlines() if not line.startswith("@")]


RC = str.maketrans("ACGT", "TGCA")


def _check_records(setup, batch, text, paired_mode=False):
    """What SAM fixes, from the records and the input bytes alone."""
    contigs = setup[0]
    by_name = dict(zip(NAMES, contigs))
    recs = _parse(text)
    primaries = {}
    for f in recs:
        qname, flag, rname, pos, mapq, cigar = f[0], int(f[1]), f[2], int(f[3]), int(f[4]), f[5]
        tags = dict((t[:2], t[5:]) for t in f[11:])
        i = int(qname[1:])
        if paired_mode:
            assert flag & 1
            read = 2 * i + (0 if flag & 64 else 1)
            assert bool(flag & 64) != bool(flag & 128)
        else:
            read = i
        seq_read = "".join("ACGT"[c] for c in batch.read(read))
        if not flag & 256:
            assert read not in primaries
            primaries[read] = f
        if flag & 4:
            assert f[9] == seq_read and cigar == "*" and mapq == 0
            continue
        m = len(seq_read)
        assert cigar == f"{m}M"
        window = by_name[rname][pos - 1:pos - 1 + m].upper()
        assert len(window) == m and set(window) <= set(b"ACGT")
        window = window.decode()
        seq = seq_read.translate(RC)[::-1] if flag & 16 else seq_read
        if not flag & 256:
            assert f[9] == seq
        assert int(tags["NM"]) == sum(a != b for a, b in zip(seq, window))
        # MD spells the reference window from SEQ
        md, rebuilt, j, num = tags["MD"], [], 0, ""
        for ch in md + "$":
            if ch.isdigit():
                num += ch
                continue
            run = int(num or 0)
            rebuilt.append(seq[j:j + run])
            j += run
            num = ""
            if ch != "$":
                rebuilt.append(ch)
                j += 1
        assert "".join(rebuilt) == window and j == m
    assert sorted(primaries) == list(range(batch.n))
    if paired_mode:
        for p in range(batch.n // 2):
            a, b = primaries[2 * p], primaries[2 * p + 1]
            for x, y in ((a, b), (b, a)):
                ry = y[2]
                assert x[6] == ("*" if ry == "*" else "=" if ry == x[2] else ry)
                assert int(x[7]) == int(y[3])
                assert bool(int(x[1]) & 8) == bool(int(y[1]) & 4)
                if not int(y[1]) & 4:
                    assert bool(int(x[1]) & 32) == bool(int(y[1]) & 16)
            assert int(a[8]) == -int(b[8])
            if int(a[1]) & 2:
                assert int(b[1]) & 2 and a[2] == b[2] and (int(a[1]) & 16) != (int(b[1]) & 16)
                assert WINDOW[0] <= abs(int(a[8])) <= WINDOW[1]


@pytest.mark.parametrize("cap,secondary", [(0, False), (0, True), (3, True)])
def test_single_end(mica, setup, single, tmp_path, cap, secondary):
    fm, ref = setup[5], setup[4]
    res = fm.align(single, cap=cap)
    got = _write(mica, tmp_path / "s.sam", ref, [(single, res, None)], secondary=secondary,
                 qname_prefix="q", command_line="bench --sam")
    want = _expected(setup, single, res, prefix="q", secondary=secondary, command_line="bench --sam")
    assert got == want
    _check_records(setup, single, got)
    flags = [int(f[1]) for f in _parse(got)]
    assert any(f & 4 for f in flags) and any(f & 16 for f in flags) and any(not f & 20 for f in flags)
    mapqs = {int(f[4]) for f in _parse(got) if not int(f[1]) & 260}
    assert mapqs == {0, 25, 37}


def test_best_stratum_result(mica, setup, single, tmp_path):
    fm, ref = setup[5], setup[4]
    res = fm.align_best_stratum(single, cap=2)
    got = _write(mica, tmp_path / "b.sam", ref, [(single, res, None)], secondary=True)
    assert got == _expected(setup, single, res, secondary=True)
    _check_records(setup, single, got)


def test_paired(mica, setup, paired, tmp_path):
    fm, ref = setup[5], setup[4]
    res = fm.align(paired, cap=0)
    tuples = oracle.pair(res, paired.lengths, *WINDOW)
    pairs = samcheck.pairs_array(tuples, mica.PAIR_DTYPE)
    got = _write(mica, tmp_path / "p.sam", ref, [(paired, res, pairs)], secondary=True, qname_prefix="p")
    assert got == _expected(setup, paired, res, pairs, prefix="p", secondary=True)
    _check_records(setup, paired, got, paired_mode=True)
    flags = [int(f[1]) for f in _parse(got) if not int(f[1]) & 256]
    assert any(f & 2 for f in flags) and any(not f & 2 for f in flags) and any(f & 8 for f in flags)
    # concordant in G but across a contig boundary or over an ambiguous base: never properly paired
    assert sum(1 for t in tuples if t[0]) > sum(1 for f in flags if f & 2) // 2


def test_batches_continue_numbering(mica, setup, single, tmp_path):
    fm, ref = setup[5], setup[4]
    res = fm.align(single)
    whole = _write(mica, tmp_path / "w.sam", ref, [(single, res, None)])
    h = single.n // 2
    a, b = single.subset(np.arange(h)), single.subset(np.arange(h, single.n))
    parts = _write(mica, tmp_path / "p.sam", ref, [(a, fm.align(a), None), (b, fm.align(b), None)])
    assert parts == whole


def test_rejects_inconsistent_input(mica, setup, single, paired, tmp_path):
    fm, ref = setup[5], setup[4]
    res = fm.align(single)
    bad = oracle.Result(res.total.copy(), res.offsets.copy(), res.hits.copy())
    bad.hits["mm"][0] = (int(bad.hits["mm"][0]) + 1) % 4          # not the hit's substitutions
    path = tmp_path / "r.sam"
    with mica.SamWriter(str(path), ref) as w:
        with pytest.raises(mica.MicaError) as e:
            w.write(single, bad)
        assert e.value.code == mica.MICA_EINVAL
    assert all(line.startswith("@") for line in open(path).read().splitlines())
    pres = fm.align(paired)
    pairs = samcheck.pairs_array(oracle.pair(pres, paired.lengths, *WINDOW), mica.PAIR_DTYPE)
    j = int(np.flatnonzero(pairs["n_concordant"] > 0)[0])
    pairs["pos_plus"][j] += 1                                      # names no listed hit
    with mica.SamWriter(str(path), ref) as w:
        with pytest.raises(mica.MicaError):
            w.write(paired, pres, pairs)
        odd = paired.subset(np.arange(3))
        with pytest.raises(mica.MicaError):
            w.write(odd, fm.align(odd), pairs[:1])
    for kw in ({"qname_prefix": "a b"}, {"qname_prefix": "@r"}, {"command_line": "x\ty"}):
        with pytest.raises(mica.MicaError):
            mica.SamWriter(str(path), ref, **kw)


def _tile(batch, res, t):
    """The batch and its result repeated t times (a batch of many chunks)."""
    class B:
        pass
    b = B()
    nw = int(batch.word_off[-1])
    b.words = np.tile(batch.words, t)
    b.word_off = np.concatenate([batch.word_off[:-1] + i * nw for i in range(t)] + [[t * nw]]).astype(np.uint64)
    b.lengths = np.tile(batch.lengths, t)
    nh = int(res.offsets[-1])
    off = np.concatenate([res.offsets[:-1] + i * nh for i in range(t)] + [[t * nh]]).astype(np.uint64)
    return b, oracle.Result(np.tile(res.total, t), off, np.tile(res.hits, t))


@pytest.mark.parametrize("paired_mode", [False, True])
def test_threads_keep_read_order(mica, setup, single, paired, tmp_path, paired_mode):
    """Batches of many 4,096-read chunks: the same text whatever the thread count."""
    fm, ref = setup[5], setup[4]
    batch = paired if paired_mode else single
    res = fm.align(batch, cap=3)
    pairs = None
    if paired_mode:
        pairs = samcheck.pairs_array(oracle.pair(res, batch.lengths, *WINDOW), mica.PAIR_DTYPE)
    t = -(-20_000 // batch.n)
    big, bres = _tile(batch, res, t)
    bpairs = None if pairs is None else np.tile(pairs, t)
    texts = []
    for threads in (1, 3, 0):
        texts.append(_write(mica, tmp_path / f"t{threads}.sam", ref, [(big, bres, bpairs)], secondary=True,
                            threads=threads))
    assert texts[0] == texts[1] == texts[2]
    one = _write(mica, tmp_path / "one.sam", ref, [(batch, res, pairs)], secondary=True)
    body = [line for line in texts[0].splitlines() if not line.startswith("@")]
    first = [line for line in one.splitlines() if not line.startswith("@")]
    assert body[:len(first)] == first                        # the first copy, numbered from 0
    assert len(body) == t * len(first)
    with pytest.raises(mica.MicaError):
        mica.SamWriter(str(tmp_path / "x.sam"), ref, threads=257)


def test_bad_read_in_a_late_chunk_writes_nothing(mica, setup, single, tmp_path):
    fm, ref = setup[5], setup[4]
    big, bres = _tile(single, fm.align(single), 40)
    j = int(bres.offsets[-1]) - 1
    bres.hits["mm"][j] = (int(bres.hits["mm"][j]) + 1) % 4      # the last listed hit
    path = tmp_path / "late.sam"
    with mica.SamWriter(str(path), ref, threads=4) as w:
        with pytest.raises(mica.MicaError):
            w.write(big, bres)
    assert all(line.startswith("@") for line in open(path).read().splitlines())


def _handworked():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "handworked_sam.txt")
    g = {"contig": [], "read": [], "sam": [], "pair": [], "psam": []}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            key, rest = line.split(" ", 1)
            g[key].append(rest)
    return g


def _result(entries, mica):
    """(codes list, result) from 'bases total pos,strand,d ...' entries."""
    codes, total, offsets, hits = [], [], [0], []
    for e in entries:
        parts = e.split()
        codes.append(np.frombuffer(parts[0].encode(), np.uint8).copy())
        total.append(int(parts[1]))
        for h in parts[2:]:
            p, s, d = h.split(",")
            hits.append((int(p), 0 if s == "+" else 1, int(d), 0))
        offsets.append(len(hits))
    for c in codes:
        c[:] = np.searchsorted(np.frombuffer(b"ACGT", np.uint8), c)
    res = oracle.Result(np.array(total, np.uint64), np.array(offsets, np.uint64),
                        np.array(hits, dtype=mica.HIT_DTYPE) if hits else np.zeros(0, mica.HIT_DTYPE))
    return codes, res


def test_handworked_records(mica, tmp_path):
    """SAM records derived by hand from the SAM specification
    (tests/golden/handworked_sam.txt): FLAG 99/147 and 73/133 pairs, TLEN,
    MD with mismatches at the end and inside, a reverse-strand secondary, a
    hit across a contig boundary left unmapped."""
    g = _handworked()
    names = [c.split()[0] for c in g["contig"]]
    seqs = [c.split()[1].encode() for c in g["contig"]]
    ref = mica.Reference.create(b"".join(seqs), [len(s) for s in seqs], names)
    header = ["@HD\tVN:1.6\tSO:unsorted"] + [f"@SQ\tSN:{n}\tLN:{len(s)}" for n, s in zip(names, seqs)] + \
             ["@PG\tID:mica-gb300\tPN:mica-gb300\tVN:1.0"]
    codes, res = _result([r.split(" ", 1)[1] for r in g["read"]], mica)
    words, off, lens = synth.pack_reads(codes)
    batch = synth.ReadBatch(words, off, lens, np.zeros(len(codes), np.uint8), np.zeros(len(codes), np.int64),
                            np.zeros(len(codes), np.uint8), np.zeros(len(codes), np.int32))
    got = _write(mica, tmp_path / "h.sam", ref, [(batch, res, None)], secondary=True, qname_prefix="r")
    assert got.splitlines() == header + [s.replace("|", "\t") for s in g["sam"]]
    mates, rows = [], []
    for p in g["pair"]:
        m1, m2, row = (x.strip() for x in p.split(" ", 1)[1].split("|"))
        mates += [m1, m2]
        rows.append(tuple(int(v) for v in row.split()) + (0,))
    codes, res = _result(mates, mica)
    words, off, lens = synth.pack_reads(codes)
    batch = synth.ReadBatch(words, off, lens, np.zeros(len(codes), np.uint8), np.zeros(len(codes), np.int64),
                            np.zeros(len(codes), np.uint8), np.zeros(len(codes), np.int32))
    pairs = np.array(rows, dtype=mica.PAIR_DTYPE)
    got = _write(mica, tmp_path / "hp.sam", ref, [(batch, res, pairs)], qname_prefix="p")
    assert got.splitlines() == header + [s.replace("|", "\t") for s in g["psam"]]
    # the restatement agrees with the hand-worked records too
    text = ref.text().decode()
    starts = [0, len(seqs[0]), len(seqs[0]) + len(seqs[1])]
    runs = [(int(s), int(s + n)) for s, n in ref.ambiguous_runs()]
    assert samcheck.sam_text(names, starts, runs, text, batch, res, pairs, prefix="p").splitlines() == \
        header + [s.replace("|", "\t") for s in g["psam"]]
