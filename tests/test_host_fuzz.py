"""Seeded fuzzing of the host-side readers and writers (no GPU): mutated
FASTQ, FASTA and reference files and corrupted results must give an error
code or a consistent result, never a crash."""
import numpy as np
import pytest

import oracle
import synth
from tests import hostlib, samcheck

ROUNDS = 150
ALPHABET = np.frombuffer(b"ACGTNacgtn@+>;\n\r \t\x00\xff-.*/12", dtype=np.uint8)


@pytest.fixture(scope="module")
def mica():
    return hostlib.mica()


def _mutate(data: bytes, rng) -> bytes:
    b = bytearray(data)
    for _ in range(int(rng.integers(1, 6))):
        op = int(rng.integers(0, 4))
        if not b:
            b.extend(rng.choice(ALPHABET, size=4).tobytes())
            continue
        j = int(rng.integers(0, len(b)))
        if op == 0:
            b[j] = int(rng.choice(ALPHABET))
        elif op == 1:
            del b[j:j + int(rng.integers(1, 20))]
        elif op == 2:
            b[j:j] = rng.choice(ALPHABET, size=int(rng.integers(1, 20))).tobytes()
        else:
            del b[j:]
    return bytes(b)


def _reads(n=40, seed=3):
    g = synth.uniform_genome(3000, seed).codes
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = rng.choice(np.array([20, 40, 90]), size=n)
    return g, synth.sample_reads(synth.Genome(g), lengths, np.full(n, 2, np.uint8), rng, subs="count")


def test_fastq_reader(mica, tmp_path):
    g, reads = _reads()
    (text,), _, _ = synth.to_fastq(reads, n_frac=0.3)
    pairs = synth.paired_reads(g, 20, seed=5, m=60, insert_mean=300.0, insert_sd=20.0)
    ptexts, _, _ = synth.to_fastq(pairs, mate_suffix=True)
    rng = np.random.Generator(np.random.PCG64(11))
    ok = bad = 0
    for r in range(ROUNDS):
        paired = r % 3 == 0
        files = list(ptexts) if paired else [text]
        files[0] = _mutate(files[0], rng)
        paths = []
        for j, t in enumerate(files):
            p = tmp_path / f"f{j}.fq"
            p.write_bytes(t)
            paths.append(str(p))
        try:
            with mica.FastqReader(*paths) as fq:
                for b in fq.batches(int(rng.integers(2, 30)), k=int(rng.integers(0, 4))):
                    assert b.paired == paired and (not paired or b.n % 2 == 0)
                    for i in range(b.n):
                        name, q, amb = b.record(i)
                        m = int(b.lengths[i])
                        assert 1 <= m <= 256 and len(q) == m and len(name) >= 1
                        assert all(0 <= a < m for a in amb) and list(amb) == sorted(set(amb))
                        assert int(b.word_off[i + 1] - b.word_off[i]) == (m + 15) // 16
            ok += 1
        except mica.MicaError as e:
            assert e.code in (mica.MICA_EIO, mica.MICA_EINVAL)
            bad += 1
    assert ok and bad


def test_fasta_and_reference_files(mica, tmp_path):
    contigs = synth.multi_contig_reference((300, 200, 500, 450), shared=0)
    text = synth.to_fasta(contigs, ["a", "b", "c", "d"], width=50)
    ref = mica.Reference.create(b"".join(contigs), [len(c) for c in contigs], ["a", "b", "c", "d"])
    ref.save(str(tmp_path / "ref.bin"))
    blob = (tmp_path / "ref.bin").read_bytes()
    rng = np.random.Generator(np.random.PCG64(12))
    outcomes = set()
    for r in range(ROUNDS):
        path = tmp_path / "m.bin"
        if r % 2:
            path.write_bytes(_mutate(text, rng))
            load = mica.Reference.from_fasta
        else:
            path.write_bytes(_mutate(blob, rng))
            load = mica.Reference.load
        try:
            x = load(str(path))
        except mica.MicaError as e:
            assert e.code in (mica.MICA_EIO, mica.MICA_EINVAL)
            outcomes.add("error")
            continue
        outcomes.add("ok")
        info, cs = x.info(), x.contigs()
        assert sum(c[2] for c in cs) == info["length"] == len(x.text())
        assert all(c[2] > 0 for c in cs) and len({c[0] for c in cs}) == len(cs)
        assert set(x.text()) <= set(b"ACGT")
        for s, ln in x.ambiguous_runs():
            assert ln > 0 and s + ln <= info["length"]
    assert outcomes == {"ok", "error"}


def test_corrupted_results(mica, tmp_path):
    g, reads = _reads(n=60, seed=7)
    ref = mica.Reference.create(synth.to_acgt_bytes(g), [1000, 1200, 800])
    good = oracle.FMIndex(g).align(reads, cap=4)
    rng = np.random.Generator(np.random.PCG64(13))
    outcomes = set()
    for r in range(ROUNDS):
        total, off, hits = good.total.copy(), good.offsets.copy(), good.hits.copy()
        for _ in range(int(rng.integers(1, 4))):
            what = int(rng.integers(0, 5))
            if what == 0 and hits.size:
                hits["pos"][int(rng.integers(0, hits.size))] = int(rng.integers(0, 2 * len(g)))
            elif what == 1 and hits.size:
                hits["strand"][int(rng.integers(0, hits.size))] = int(rng.integers(0, 4))
            elif what == 2 and hits.size:
                hits["mm"][int(rng.integers(0, hits.size))] = int(rng.integers(0, 256))
            elif what == 3:
                total[int(rng.integers(0, total.size))] = int(rng.integers(0, 6))
            else:
                j = int(rng.integers(1, off.size - 1))
                off[j] = min(int(off[-1]), int(off[j]) + int(rng.integers(-2, 3)) if int(off[j]) > 1 else 0)
        bad = oracle.Result(total, off, hits)
        for call in ("filter", "sam"):
            try:
                if call == "filter":
                    ref.filter(bad, reads.lengths)
                else:
                    with mica.SamWriter(str(tmp_path / "c.sam"), ref, threads=int(rng.integers(0, 4))) as w:
                        w.write(reads, bad)
                outcomes.add("ok")
            except mica.MicaError as e:
                assert e.code == mica.MICA_EINVAL
                outcomes.add("error")
    assert outcomes == {"ok", "error"}
    pairs = synth.paired_reads(g, 30, seed=8, m=60, insert_mean=300.0, insert_sd=20.0)
    pres = oracle.FMIndex(g).align(pairs)
    rows = samcheck.pairs_array(oracle.pair(pres, pairs.lengths, 200, 400), mica.PAIR_DTYPE)
    for r in range(40):
        bad_rows = rows.copy()
        j = int(rng.integers(0, rows.size))
        field = ["n_concordant", "n_best", "pos_plus", "pos_minus", "plus_mate"][int(rng.integers(0, 5))]
        bad_rows[field][j] = int(rng.integers(0, 2 ** 8))
        try:
            with mica.SamWriter(str(tmp_path / "p.sam"), ref) as w:
                w.write(pairs, pres, bad_rows)
        except mica.MicaError as e:
            assert e.code == mica.MICA_EINVAL
