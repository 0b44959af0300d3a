"""References of several contigs with ambiguous bases (host-side, no GPU).

The oracle's reference rule (oracle.reference_concat / reference_filter) is
pinned against the published SplitMix64 outputs and against a brute-force
Hamming scan of each contig's own bytes; the library's mica_reference_* calls
(C++, no CUDA) are compared with the oracle on the same inputs.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import hostlib, refcheck

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "splitmix64.txt")
NAMES = ["chr1", "chr2", "chrUn_1", "chrM"]


@pytest.fixture(scope="module")
def mica():
    return hostlib.mica()


@pytest.fixture(scope="module")
def contigs():
    return synth.multi_contig_reference()


@pytest.fixture(scope="module")
def concat(contigs):
    return oracle.reference_concat(contigs)


@pytest.fixture(scope="module")
def reads(concat):
    """Reads of G, half of them drawn around contig boundaries and ambiguous
    runs so that the search finds windows the reference rule must drop."""
    g, starts, runs = concat
    regions = [(max(0, s - 160), min(len(g), s + 160), "boundary") for s in starts[1:-1]]
    regions += [(max(0, s - 160), min(len(g), e + 160), "ambiguous") for s, e in runs]
    rng = np.random.Generator(np.random.PCG64(synth.SEED_REFERENCE_READS))
    n = 400
    lengths = rng.choice(np.array([50, 100, 150]), size=n)
    k = rng.integers(0, 3, size=n, dtype=np.uint8)
    return synth.sample_reads(synth.Genome(g, regions), lengths, k, rng, subs="count", max_subs=2,
                              repeat_frac=0.5)


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            state, outs = line.split(":")
            vals[int(state)] = [int(x) for x in outs.split()]
    return vals


def test_splitmix64_matches_published_outputs():
    for state, outs in _golden().items():
        got, s = [], state
        for _ in outs:
            got.append(oracle.splitmix64(s))
            s = (s + 0x9E3779B97F4A7C15) % (1 << 64)
        assert got == outs


def test_oracle_concat_by_definition(contigs, concat):
    g, starts, runs = concat
    raw = np.frombuffer(b"".join(contigs), dtype=np.uint8)
    assert starts == list(np.cumsum([0] + [len(c) for c in contigs]))
    amb = ~np.isin(raw, np.frombuffer(b"ACGTacgt", dtype=np.uint8))
    # runs are the maximal runs of ambiguous coordinates
    mask = np.zeros(len(raw), dtype=bool)
    for s, e in runs:
        mask[s:e] = True
    assert (mask == amb).all()
    assert all(runs[j][1] < runs[j + 1][0] for j in range(len(runs) - 1))
    upper = raw & ~np.uint8(0x20)
    assert (np.frombuffer(b"ACGT", dtype=np.uint8)[g][~amb] == upper[~amb]).all()
    for j in np.flatnonzero(amb):
        assert g[j] == oracle.splitmix64(int(j)) >> 62


def test_oracle_filtered_search_equals_contig_scan(contigs, concat, reads):
    """Search over G then drop the windows off the reference == brute force on
    each contig's own bytes (which never sees the replaced bases)."""
    g, starts, runs = concat
    res, dropped = oracle.reference_filter(oracle.FMIndex(g).align(reads), reads.lengths, starts, runs)
    assert dropped > 0
    for i in range(reads.n):
        want = refcheck.contig_hamming_hits(contigs, reads.read(i), int(reads.k[i]))
        assert res.as_tuples(i) == want, i
        assert int(res.total[i]) == len(want)


def test_library_reference_matches_oracle(mica, contigs, concat):
    g, starts, runs = concat
    ref = mica.Reference.create(b"".join(contigs), [len(c) for c in contigs], NAMES)
    assert ref.text() == synth.to_acgt_bytes(g)
    assert ref.contigs() == [(n, starts[i], starts[i + 1] - starts[i]) for i, n in enumerate(NAMES)]
    assert [(int(s), int(s + ln)) for s, ln in ref.ambiguous_runs()] == runs
    info = ref.info()
    assert info["length"] == len(g) and info["n_contigs"] == 4
    assert info["ambiguous_bases"] == sum(e - s for s, e in runs)


@pytest.mark.parametrize("cap", [0, 3])
def test_library_filter_matches_oracle(mica, contigs, concat, reads, cap):
    g, starts, runs = concat
    ref = mica.Reference.create(b"".join(contigs), [len(c) for c in contigs], NAMES)
    full = oracle.FMIndex(g).align(reads, cap=cap)
    want, wd = oracle.reference_filter(full, reads.lengths, starts, runs)
    got, gd = ref.filter(full, reads.lengths)
    assert gd == wd > 0
    assert (got.offsets == want.offsets).all() and (got.total == want.total).all()
    assert (got.hits == want.hits).all()


def test_locate(mica, contigs, concat):
    g, starts, runs = concat
    ref = mica.Reference.create(b"".join(contigs), [len(c) for c in contigs], NAMES)
    rng = np.random.Generator(np.random.PCG64(5))
    m = 100
    pos = rng.integers(0, len(g) - m + 1, size=3000)
    pos = np.concatenate([pos, np.array(starts[1:-1]) - m, np.array(starts[1:-1]) - m + 1, [0, len(g) - m]])
    contig, local = ref.locate(pos, m)
    for p, c, l in zip(pos, contig, local):
        if oracle.on_reference(int(p), m, starts, runs):
            assert c >= 0 and starts[c] <= p < starts[c + 1] and l == p - starts[c]
        else:
            assert c == -1 and l == 0
    with pytest.raises(mica.MicaError):
        ref.locate([len(g) - m + 1], m)     # ends past G
    with pytest.raises(mica.MicaError):
        ref.locate([0], 0)                  # empty window


def test_filter_rejects_bad_input_and_changes_nothing(mica, contigs, concat, reads):
    g, starts, runs = concat
    ref = mica.Reference.create(b"".join(contigs), [len(c) for c in contigs], NAMES)
    res = oracle.FMIndex(g).align(reads)
    bad = oracle.Result(res.total.copy(), res.offsets.copy(), res.hits.copy())
    i = int(np.flatnonzero(np.diff(bad.offsets.astype(np.int64)) > 0)[0])
    bad.hits["pos"][int(bad.offsets[i])] = len(g) - 10      # ends past G
    with pytest.raises(mica.MicaError) as e:
        ref.filter(bad, reads.lengths)
    assert e.value.code == mica.MICA_EINVAL
    short = oracle.Result(res.total.copy(), res.offsets.copy(), res.hits.copy())
    short.total[i] = 0                                        # more listed than total
    with pytest.raises(mica.MicaError):
        ref.filter(short, reads.lengths)


def test_fasta_reader(mica, contigs, tmp_path):
    for width, crlf in ((60, False), (77, True), (10 ** 6, False)):
        text = b";comment line\n\n" + synth.to_fasta(contigs, NAMES, width=width, crlf=crlf)
        path = tmp_path / f"ref_{width}.fa"
        path.write_bytes(text)
        ref = mica.Reference.from_fasta(str(path))
        mem = mica.Reference.create(b"".join(contigs), [len(c) for c in contigs], NAMES)
        assert ref.text() == mem.text()
        assert ref.contigs() == mem.contigs()
        assert (ref.ambiguous_runs() == mem.ambiguous_runs()).all()


@pytest.mark.parametrize("text", [
    b"ACGT\n>x\nACGT\n",             # bytes before the first record
    b">x\nACGT\n>y\n>z\nAC\n",       # empty record
    b">x\nAC-GT\n",                  # a gap character
    b">x\nACGT\n>x\nACGT\n",         # repeated name
    b"> x\nACGT\n",                  # empty name
    b">x(1)\nACGT\n",                # not a SAM reference name
    b"",                             # no record
])
def test_fasta_reader_rejects_malformed(mica, tmp_path, text):
    path = tmp_path / "bad.fa"
    path.write_bytes(text)
    with pytest.raises(mica.MicaError) as e:
        mica.Reference.from_fasta(str(path))
    assert e.value.code == mica.MICA_EIO


def test_create_rejections(mica):
    with pytest.raises(mica.MicaError):
        mica.Reference.create(b"ACGTACGT", [4, 0, 4])            # empty contig
    with pytest.raises(mica.MicaError):
        mica.Reference.create(b"ACGTACGT", [4, 3])               # lengths do not sum
    with pytest.raises(mica.MicaError):
        mica.Reference.create(b"ACGTACGT", [4, 4], ["a", "a"])   # repeated name
    with pytest.raises(mica.MicaError):
        mica.Reference.create(b"ACGTACGT", [4, 4], ["a", "*b"])  # invalid first character
    r = mica.Reference.create(b"ACGTACGT", [4, 4])
    assert [c[0] for c in r.contigs()] == ["contig1", "contig2"]


def test_save_load_roundtrip_and_corruption(mica, contigs, tmp_path):
    ref = mica.Reference.create(b"".join(contigs), [len(c) for c in contigs], NAMES)
    path = str(tmp_path / "ref.bin")
    ref.save(path)
    back = mica.Reference.load(path)
    assert back.text() == ref.text() and back.contigs() == ref.contigs()
    assert (back.ambiguous_runs() == ref.ambiguous_runs()).all()
    blob = open(path, "rb").read()
    for bad in (blob[:-1], blob + b"\0", b"X" + blob[1:]):
        with open(path, "wb") as f:
            f.write(bad)
        with pytest.raises(mica.MicaError) as e:
            mica.Reference.load(path)
        assert e.value.code == mica.MICA_EIO
