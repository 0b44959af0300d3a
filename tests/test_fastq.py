"""Reads from FASTQ and ambiguous read bases (host-side, no GPU).

The library's FASTQ reader is checked against the generator's own record of
what it wrote (bases, names, qualities, ambiguous offsets, the documented
stand-in base); the N rule (oracle.n_filter) is pinned by a brute-force
Hamming scan in which an ambiguous base equals no base, and the library's
mica_read_batch_filter_n equals the oracle's; SAM records of a batch carry
its names, qualities and N."""
import numpy as np
import pytest

import oracle
import synth
from tests import hostlib, refcheck, samcheck

WINDOW = (200, 600)


@pytest.fixture(scope="module")
def mica():
    return hostlib.mica()


@pytest.fixture(scope="module")
def genome():
    return synth.uniform_genome(30_000, synth.SEED_FASTQ).codes


@pytest.fixture(scope="module")
def single(genome):
    rng = np.random.Generator(np.random.PCG64(synth.SEED_FASTQ + 1))
    n = 600
    lengths = rng.choice(np.array([30, 60, 100, 150]), size=n)
    k = np.full(n, 2, dtype=np.uint8)
    return synth.sample_reads(synth.Genome(genome), lengths, k, rng, subs="count", max_subs=2)


def _read_all(mica, paths, size, k=2):
    with mica.FastqReader(*paths) as fq:
        return list(fq.batches(size, k))


def _write(tmp_path, texts):
    paths = []
    for j, t in enumerate(texts):
        p = tmp_path / f"r{j + 1}.fq"
        p.write_bytes(t)
        paths.append(str(p))
    return paths


@pytest.mark.parametrize("crlf,size", [(False, 1000), (True, 37)])
def test_reader_matches_what_was_written(mica, single, tmp_path, crlf, size):
    texts, amb, quals = synth.to_fastq(single, crlf=crlf)
    batches = _read_all(mica, _write(tmp_path, texts), size, k=3)
    assert sum(b.n for b in batches) == single.n
    assert all(b.n == size for b in batches[:-1])
    i = 0
    for b in batches:
        assert not b.paired and (b.k == 3).all()
        for j in range(b.n):
            name, q, a = b.record(j)
            assert name == f"read{i}" and q == quals[i] and list(a) == amb[i]
            assert int(b.lengths[j]) == int(single.lengths[i])
            got, want = b.read(j), single.read(i)
            keep = np.ones(len(want), dtype=bool)
            keep[amb[i]] = False
            assert (got[keep] == want[keep]).all()
            for off in amb[i]:      # the documented stand-in base
                assert got[off] == oracle.splitmix64((i << 8) + off) >> 62
            i += 1
    assert sum(b.n_ambiguous_reads for b in batches) == sum(1 for a in amb if a)


def test_paired_files(mica, genome, tmp_path):
    pairs = synth.paired_reads(genome, 120, seed=synth.SEED_FASTQ + 2, m=100, insert_mean=350.0, insert_sd=40.0)
    texts, amb, quals = synth.to_fastq(pairs, mate_suffix=True)
    batches = _read_all(mica, _write(tmp_path, texts), 51)      # rounded down to 50 reads
    assert [b.n for b in batches] == [50] * 4 + [40]
    i = 0
    for b in batches:
        assert b.paired
        for j in range(b.n):
            name, q, a = b.record(j)
            assert name == f"frag{i // 2}" and q == quals[i] and list(a) == amb[i]
            i += 1


@pytest.mark.parametrize("text,code", [
    (b"read\nACGT\n+\nIIII\n", "EIO"),            # no '@'
    (b"@r\nACGT\nIIII\n", "EIO"),                 # no '+' line
    (b"@r\nACGT\n+\nIII\n", "EIO"),               # qualities shorter than the bases
    (b"@r\nAC-T\n+\nIIII\n", "EIO"),              # a gap character
    (b"@r@1\nACGT\n+\nIIII\n", "EIO"),            # '@' inside the name
    (b"@r\nACGT\n+\nII\x7fI\n", "EIO"),           # a quality outside 33..126
    (b"@r\nACGT\n", "EIO"),                       # truncated record
    (b"@r\n\n+\n\n", "EINVAL"),                   # an empty read
    (b"@r\n" + b"A" * 257 + b"\n+\n" + b"I" * 257 + b"\n", "EINVAL"),
])
def test_reader_rejects_malformed(mica, tmp_path, text, code):
    p = tmp_path / "bad.fq"
    p.write_bytes(text)
    with mica.FastqReader(str(p)) as fq:
        with pytest.raises(mica.MicaError) as e:
            fq.read(10)
    assert e.value.code == getattr(mica, "MICA_" + code)


def test_reader_rejects_bad_mates_and_arguments(mica, tmp_path):
    a = tmp_path / "a.fq"
    b = tmp_path / "b.fq"
    a.write_bytes(b"@x/1\nACGT\n+\nIIII\n@y/1\nACGT\n+\nIIII\n")
    b.write_bytes(b"@x/2\nACGT\n+\nIIII\n")
    with mica.FastqReader(str(a), str(b)) as fq:
        assert fq.read(2).n == 2
        with pytest.raises(mica.MicaError):
            fq.read(2)                                   # mate files of different lengths
    b.write_bytes(b"@x/2\nACGT\n+\nIIII\n@z/2\nACGT\n+\nIIII\n")
    with mica.FastqReader(str(a), str(b)) as fq:
        with pytest.raises(mica.MicaError):
            fq.read(4)                                   # mates' names differ
        with pytest.raises(mica.MicaError):
            fq.read(1)                                   # fewer than one pair
    with mica.FastqReader(str(a)) as fq:
        with pytest.raises(mica.MicaError):
            fq.read(10, k=4)
    with pytest.raises(mica.MicaError):
        mica.FastqReader(str(tmp_path / "missing.fq"))


def _batch_with_n(mica, single, tmp_path):
    texts, amb, quals = synth.to_fastq(single, n_frac=0.5, max_n=2)
    (b,) = _read_all(mica, _write(tmp_path, texts), 10_000)
    return b, amb


def test_n_rule_oracle_equals_brute_force(mica, genome, single, tmp_path):
    b, amb = _batch_with_n(mica, single, tmp_path)
    res = oracle.FMIndex(genome).align(b)
    reads = [b.read(i) for i in range(b.n)]
    got, dropped = oracle.n_filter(res, reads, amb, b.k, genome)
    assert dropped > 0
    for i in range(b.n):
        r = reads[i].astype(np.int16)
        r[amb[i]] = 255
        want = refcheck.hamming_hits_n(genome, r, int(b.k[i]))
        assert got.as_tuples(i) == want, i
        assert int(got.total[i]) == len(want)


@pytest.mark.parametrize("cap", [0, 2])
def test_library_n_filter_equals_oracle(mica, genome, single, tmp_path, cap):
    b, amb = _batch_with_n(mica, single, tmp_path)
    ref = mica.Reference.create(synth.to_acgt_bytes(genome), [len(genome)])
    res = oracle.FMIndex(genome).align(b, cap=cap)
    want, wd = oracle.n_filter(res, [b.read(i) for i in range(b.n)], amb, b.k, genome)
    got, gd = b.filter_n(ref, res)
    assert gd == wd
    assert (got.offsets == want.offsets).all() and (got.total == want.total).all()
    assert (got.hits[["pos", "strand", "mm"]] == want.hits[["pos", "strand", "mm"]]).all()
    again, gd2 = b.filter_n(ref, got)                     # idempotent
    assert gd2 == 0 and (again.hits == got.hits).all()
    bad = oracle.Result(res.total.copy(), res.offsets.copy(), res.hits.copy())
    i = next(i for i in range(b.n) if amb[i] and res.offsets[i + 1] > res.offsets[i])
    h = int(bad.offsets[i])
    bad.hits["mm"][h] = 200                                  # neither d nor d' (reads of <= 150 bases)
    with pytest.raises(mica.MicaError):
        b.filter_n(ref, bad)


def test_sam_of_a_batch(mica, genome, single, tmp_path):
    b, amb = _batch_with_n(mica, single, tmp_path)
    ref = mica.Reference.create(synth.to_acgt_bytes(genome), [len(genome)], ["chrS"])
    res = oracle.FMIndex(genome).align(b, cap=3)
    info = [b.record(i) for i in range(b.n)]
    text = synth.to_acgt_bytes(genome).decode()
    want = samcheck.sam_text(["chrS"], [0, len(genome)], [], text, b, res, secondary=True,
                             records=[(n, q, list(a), int(k)) for (n, q, a), k in zip(info, b.k)])
    for hits in (res, b.filter_n(ref, res)[0]):           # before or after the N filter
        path = tmp_path / "batch.sam"
        with mica.SamWriter(str(path), ref, secondary=True) as w:
            w.write_batch(b, hits)
        assert open(path).read() == want
    recs = [line.split("\t") for line in want.splitlines() if not line.startswith("@")]
    assert any("N" in f[9] for f in recs if not int(f[1]) & 4)
    for f in recs:
        if int(f[1]) & 256:
            continue
        name, q, a = info[int(f[0][4:])]
        assert f[0] == name
        assert f[10] == (q[::-1] if int(f[1]) & 16 else q)


def test_sam_of_a_paired_batch(mica, genome, tmp_path):
    pairs = synth.paired_reads(genome, 200, seed=synth.SEED_FASTQ + 3, m=100, insert_mean=350.0, insert_sd=40.0)
    texts, amb, quals = synth.to_fastq(pairs, mate_suffix=True, n_frac=0.3)
    (b,) = _read_all(mica, _write(tmp_path, texts), 10_000)
    ref = mica.Reference.create(synth.to_acgt_bytes(genome), [len(genome)], ["chrS"])
    fres, _ = b.filter_n(ref, oracle.FMIndex(genome).align(b))
    res = oracle.Result(fres.total, fres.offsets, fres.hits)
    pr = samcheck.pairs_array(oracle.pair(res, b.lengths, *WINDOW), mica.PAIR_DTYPE)
    records = [(n, q, list(a), int(k)) for (n, q, a), k in zip((b.record(i) for i in range(b.n)), b.k)]
    text = synth.to_acgt_bytes(genome).decode()
    for pairs_rows in (pr, None):
        path = tmp_path / "pairs.sam"
        with mica.SamWriter(str(path), ref) as w:
            w.write_batch(b, res, pairs_rows)
        want = samcheck.sam_text(["chrS"], [0, len(genome)], [], text, b, res,
                                 pr if pairs_rows is not None else samcheck.no_pairs(b.n // 2, mica.PAIR_DTYPE),
                                 records=records)
        assert open(path).read() == want
    flags = [int(line.split("\t")[1]) for line in want.splitlines() if not line.startswith("@")]
    assert all(f & 1 for f in flags)
