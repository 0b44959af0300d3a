"""Seeded synthetic genomes and reads for the k-mismatch read search.

This module only makes inputs: it holds none of the search arithmetic, and
both the CPU oracle (``oracle/``) and the CUDA library are fed from it.  The
paper's experiments (Section 3, Table 1 and Table 2) use real human data
(YH PE150/PE100, 1000 Genomes lanes) that are not available here; the
generators below produce stand-ins with the same read lengths (100/150 bp),
the paper's batch size of about a million reads (Section 2), and genomes whose
repeat structure makes the backtracking work uneven across reads.

Encoding: a genome or read is a ``uint8`` array of base codes A=0, C=1, G=2,
T=3.  A batch of reads is packed 2 bits per base, 16 bases per ``uint32`` word,
least-significant bits first; read ``i`` starts at word ``word_off[i]``.

Every generator draws from ``numpy.random.Generator(PCG64(seed))`` only.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)

# Seeds of the five workloads (genome, reads, slice ...).
SEED_GENOME_1M = 1
SEED_READS_1M = 11
SEED_SLICE_10K = 12
SEED_GENOME_64M = 2
SEED_READS_64M = 21
SEED_READS_UNEVEN = 31
SEED_GENOME_HUMAN = 4
SEED_DONOR_HUMAN = 41
SEED_READS_HUMAN = 42
SEED_ARRIVALS = 51
SEED_READS_SERVE = 52
SEED_REFERENCE = 61
SEED_REFERENCE_READS = 62


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def to_acgt_bytes(codes: np.ndarray) -> bytes:
    """Base codes 0..3 -> ASCII 'ACGT' bytes (the library's genome input)."""
    return ACGT[np.asarray(codes, dtype=np.uint8)].tobytes()


def opposite_strand(codes: np.ndarray) -> np.ndarray:
    """The other strand of a DNA segment, read 5'->3' (used to draw reads
    from the minus strand and to copy repeats in reverse orientation)."""
    return (3 - np.asarray(codes, dtype=np.uint8))[::-1].copy()


def substitute(codes: np.ndarray, where: np.ndarray, rng: np.random.Generator) -> None:
    """In place: replace the bases at ``where`` by one of the three other bases,
    uniformly."""
    if len(where) == 0:
        return
    shift = rng.integers(1, 4, size=len(where), dtype=np.uint8)
    codes[where] = (codes[where] + shift) & 3


# --------------------------------------------------------------------------
# Genomes
# --------------------------------------------------------------------------

@dataclass
class Genome:
    codes: np.ndarray                      # uint8 base codes, length N
    regions: list = field(default_factory=list)  # (start, end, kind) of planted repeats

    @property
    def n(self) -> int:
        return int(self.codes.shape[0])


def uniform_genome(n: int, seed: int) -> Genome:
    """i.i.d. uniform A/C/G/T genome of length ``n``."""
    return Genome(_rng(seed).integers(0, 4, size=n, dtype=np.uint8))


def repeat_genome(n: int, seed: int, *, copy_frac: float = 0.05,
                  copy_len=(1_000, 10_000), copy_div: float = 0.01,
                  tandem_frac: float = 0.01, unit_len=(2, 50),
                  array_len=(100, 5_000), tandem_div: float = 0.0) -> Genome:
    """Genome with interspersed copies and tandem arrays.

    1. i.i.d. uniform base sequence;
    2. segments of length uniform in ``copy_len`` copied from a random source
       position to a random destination, in random orientation, each copied
       base substituted with probability ``copy_div``, until ``copy_frac`` of
       the length has been overwritten;
    3. tandem arrays: a random unit of length uniform in ``unit_len`` repeated
       to an array length uniform in ``array_len`` (each base substituted with
       probability ``tandem_div``), until ``tandem_frac`` of the length is
       covered.
    """
    rng = _rng(seed)
    g = rng.integers(0, 4, size=n, dtype=np.uint8)
    regions = []
    budget = int(copy_frac * n)
    while budget > 0:
        ln = int(rng.integers(copy_len[0], copy_len[1] + 1))
        ln = min(ln, n // 4)
        src = int(rng.integers(0, n - ln + 1))
        dst = int(rng.integers(0, n - ln + 1))
        seg = g[src:src + ln].copy()
        if rng.integers(0, 2):
            seg = opposite_strand(seg)
        hit = np.flatnonzero(rng.random(ln) < copy_div)
        substitute(seg, hit, rng)
        g[dst:dst + ln] = seg
        regions.append((dst, dst + ln, "copy"))
        budget -= ln
    budget = int(tandem_frac * n)
    while budget > 0:
        u = int(rng.integers(unit_len[0], unit_len[1] + 1))
        ln = int(rng.integers(array_len[0], array_len[1] + 1))
        ln = min(ln, n // 4)
        unit = rng.integers(0, 4, size=u, dtype=np.uint8)
        arr = np.resize(unit, ln)
        if tandem_div > 0:
            hit = np.flatnonzero(rng.random(ln) < tandem_div)
            substitute(arr, hit, rng)
        dst = int(rng.integers(0, n - ln + 1))
        g[dst:dst + ln] = arr
        regions.append((dst, dst + ln, "tandem"))
        budget -= ln
    return Genome(g, regions)


# --------------------------------------------------------------------------
# Reads
# --------------------------------------------------------------------------

@dataclass
class ReadBatch:
    """A batch of reads in the library's packed layout, with ground truth."""
    words: np.ndarray        # uint32 packed bases
    word_off: np.ndarray     # uint64, n+1 word offsets
    lengths: np.ndarray      # uint16 read lengths
    k: np.ndarray            # uint8 per-read mismatch budget
    origin: np.ndarray       # int64 sampled origin (leftmost forward coordinate)
    strand: np.ndarray       # uint8 0 = forward, 1 = reverse complement
    n_subs: np.ndarray       # int32 substitutions applied to the read

    @property
    def n(self) -> int:
        return int(self.lengths.shape[0])

    def read(self, i: int) -> np.ndarray:
        """Unpacked base codes of read ``i``."""
        m = int(self.lengths[i])
        w = self.words[int(self.word_off[i]):int(self.word_off[i + 1])]
        return unpack_words(w, m)

    def subset(self, idx) -> "ReadBatch":
        """The reads `idx` (in that order) as a batch of their own."""
        idx = np.asarray(idx, dtype=np.int64)
        off = self.word_off.astype(np.int64)
        starts, counts = off[idx], off[idx + 1] - off[idx]
        new_off = np.zeros(len(idx) + 1, dtype=np.uint64)
        np.cumsum(counts, out=new_off[1:])
        total = int(new_off[-1])
        src = np.repeat(starts - new_off[:-1].astype(np.int64), counts) + np.arange(total, dtype=np.int64)
        return ReadBatch(self.words[src].copy(), new_off, self.lengths[idx].copy(), self.k[idx].copy(),
                         self.origin[idx].copy(), self.strand[idx].copy(), self.n_subs[idx].copy())


def unpack_words(words: np.ndarray, m: int) -> np.ndarray:
    w = np.asarray(words, dtype=np.uint32)
    shifts = (2 * np.arange(16, dtype=np.uint32))
    bases = ((w[:, None] >> shifts[None, :]) & 3).astype(np.uint8).reshape(-1)
    return bases[:m].copy()


def pack_reads(reads) -> tuple:
    """List of uint8 code arrays -> (words uint32, word_off uint64[n+1], lengths uint16)."""
    n = len(reads)
    lens = np.fromiter((len(r) for r in reads), dtype=np.int64, count=n)
    nw = (lens + 15) // 16
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(nw, out=off[1:])
    words = np.zeros(int(off[-1]), dtype=np.uint32)
    # group reads of equal length and pack each group with array operations
    for m in np.unique(lens):
        idx = np.flatnonzero(lens == m)
        mat = np.stack([reads[i] for i in idx]).astype(np.uint32)
        _pack_group(words, off, idx, mat)
    return words, off, lens.astype(np.uint16)


def _pack_group(words, off, idx, mat):
    m = mat.shape[1]
    w = (m + 15) // 16
    pad = np.zeros((mat.shape[0], w * 16), dtype=np.uint32)
    pad[:, :m] = mat
    pad = pad.reshape(mat.shape[0], w, 16) << (2 * np.arange(16, dtype=np.uint32))
    packed = np.bitwise_or.reduce(pad, axis=2)
    dst = off[idx].astype(np.int64)[:, None] + np.arange(w)[None, :]
    words[dst] = packed


def sample_reads(genome: Genome, lengths: np.ndarray, k: np.ndarray, rng: np.random.Generator, *,
                 subs: str, sub_rate: float = 0.01, max_subs: int = 2,
                 repeat_frac: float = 0.0, origin_limit: int | None = None) -> ReadBatch:
    """Draw reads from ``genome``.

    Origin uniform in [0, N-m] (or, for a fraction ``repeat_frac`` of reads,
    uniform inside a planted repeat region chosen with probability proportional
    to its length); strand a fair coin; then substitutions:
    ``subs == "count"``: a number uniform in {0..max_subs} at distinct uniform
    positions; ``subs == "rate"``: each base i.i.d. with probability ``sub_rate``.
    The replacement base is uniform among the three others.
    """
    g = genome.codes
    n_total = genome.n if origin_limit is None else origin_limit
    n = len(lengths)
    lengths = np.asarray(lengths, dtype=np.int64)
    origin = (rng.random(n) * (n_total - lengths + 1)).astype(np.int64)
    if repeat_frac > 0 and genome.regions:
        reg = np.array([(a, b) for a, b, _ in genome.regions], dtype=np.int64)
        w = (reg[:, 1] - reg[:, 0]).astype(np.float64)
        pick = rng.random(n) < repeat_frac
        ridx = rng.choice(len(reg), size=int(pick.sum()), p=w / w.sum())
        a = reg[ridx, 0]
        b = np.maximum(reg[ridx, 1] - lengths[pick], a)
        o = a + (rng.random(len(ridx)) * (b - a + 1)).astype(np.int64)
        origin[pick] = np.minimum(o, n_total - lengths[pick])
    strand = rng.integers(0, 2, size=n, dtype=np.uint8)
    n_subs = np.zeros(n, dtype=np.int32)
    nw = (lengths + 15) // 16
    off = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(nw, out=off[1:])
    words = np.zeros(int(off[-1]), dtype=np.uint32)
    for m in np.unique(lengths):
        idx = np.flatnonzero(lengths == m)
        mat = g[origin[idx][:, None] + np.arange(m)[None, :]]
        rev = strand[idx] == 1
        mat[rev] = (3 - mat[rev])[:, ::-1]
        if subs == "count":
            cnt = rng.integers(0, max_subs + 1, size=len(idx))
            for j, c in enumerate(cnt):
                if c:
                    pos = rng.choice(m, size=int(c), replace=False)
                    substitute(mat[j], pos, rng)
            n_subs[idx] = cnt
        elif subs == "rate":
            hit = rng.random(mat.shape) < sub_rate
            flat = mat.reshape(-1)
            substitute(flat, np.flatnonzero(hit.reshape(-1)), rng)
            mat = flat.reshape(mat.shape)
            n_subs[idx] = hit.sum(axis=1)
        else:
            raise ValueError(subs)
        _pack_group(words, off, idx, mat.astype(np.uint32))
    lens = lengths.astype(np.uint16)
    return ReadBatch(words, off, lens, np.asarray(k, dtype=np.uint8), origin, strand, n_subs)


# --------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------

def genome_1m() -> Genome:
    """Small case: i.i.d. uniform genome of 1 Mbp."""
    return uniform_genome(1_000_000, SEED_GENOME_1M)


def reads_1m(genome: Genome, n: int = 10_000) -> ReadBatch:
    """10,000 reads of 100 bp, 0-2 substitutions at distinct uniform positions, k = 2."""
    rng = _rng(SEED_READS_1M)
    return sample_reads(genome, np.full(n, 100), np.full(n, 2), rng, subs="count", max_subs=2)


def slice_10k(genome: Genome, n: int = 1_000, m: int = 100) -> tuple:
    """Brute-force slice: the first 10,000 bp of the 1 Mbp genome as a genome of
    its own, and 1,000 reads drawn from it with 0-2 substitutions."""
    g = Genome(genome.codes[:10_000].copy())
    rng = _rng(SEED_SLICE_10K)
    return g, sample_reads(g, np.full(n, m), np.full(n, 2), rng, subs="count", max_subs=2)


def genome_64m(n: int = 1 << 26) -> Genome:
    """Repeat genome of 64 Mbp: 5% copies of 1-10 kbp at 1% divergence, 1% tandem
    arrays (unit 2-50 bp, array 100-5,000 bp, exact copies)."""
    return repeat_genome(n, SEED_GENOME_64M)


def reads_64m(genome: Genome, n: int = 1_000_000, m: int = 150, seed: int = SEED_READS_64M) -> ReadBatch:
    """1M reads of 150 bp with 1% i.i.d. substitution error, k = 2."""
    rng = _rng(seed)
    return sample_reads(genome, np.full(n, m), np.full(n, 2), rng, subs="rate", sub_rate=0.01)


UNEVEN_LENGTHS = (50, 100, 150, 250)


def reads_uneven(genome: Genome, n: int = 1_000_000) -> ReadBatch:
    """1M reads, length uniform over {50, 100, 150, 250}, k uniform over {0..3},
    30% drawn from inside planted repeats, 1% substitution error."""
    rng = _rng(SEED_READS_UNEVEN)
    lengths = np.asarray(UNEVEN_LENGTHS)[rng.integers(0, 4, size=n)]
    k = rng.integers(0, 4, size=n).astype(np.uint8)
    return sample_reads(genome, lengths, k, rng, subs="rate", sub_rate=0.01, repeat_frac=0.30)


# --------------------------------------------------------------------------
# Human-scale genome and paired reads
# --------------------------------------------------------------------------

HUMAN_LEN = 3_100_000_000


def _plant(g, seg, dst, rev):
    if rev:
        seg = opposite_strand(seg)
    g[dst:dst + len(seg)] = seg


def human_genome(n: int = HUMAN_LEN, seed: int = SEED_GENOME_HUMAN) -> Genome:
    """About 45% repeats over an i.i.d. base:

    * 300 bp families: 50 consensus sequences; copies with per-copy
      divergence uniform in 10-15%, random orientation, covering 15%;
    * 6 kbp families: 20 consensus sequences; copies at 5% divergence,
      full length or 5'-truncated (half each; truncated length uniform in
      300-6,000 bp, the 3' end kept), covering 25%;
    * tandem arrays: unit 2-50 bp, array 100-20,000 bp, per-array divergence
      uniform in 1-5%, covering 5%.
    Later plantings overwrite earlier ones where they overlap.
    """
    rng = _rng(seed)
    g = rng.integers(0, 4, size=n, dtype=np.uint8)
    regions = []
    # 300 bp families
    fam = rng.integers(0, 4, size=(50, 300), dtype=np.uint8)
    total = int(0.15 * n)
    done = 0
    while done < total:
        c = min(100_000, (total - done) // 300 + 1)
        f = rng.integers(0, 50, size=c)
        div = rng.uniform(0.10, 0.15, size=c)
        mat = fam[f].copy()
        hit = rng.random(mat.shape) < div[:, None]
        shift = rng.integers(1, 4, size=mat.shape, dtype=np.uint8)
        mat = np.where(hit, (mat + shift) & 3, mat).astype(np.uint8)
        rev = rng.integers(0, 2, size=c)
        dst = rng.integers(0, n - 300, size=c)
        for j in range(c):
            _plant(g, mat[j], int(dst[j]), rev[j])
            regions.append((int(dst[j]), int(dst[j]) + 300, "fam300"))
        done += 300 * c
    # 6 kbp families
    fam = rng.integers(0, 4, size=(20, 6000), dtype=np.uint8)
    total = int(0.25 * n)
    done = 0
    while done < total:
        f = int(rng.integers(0, 20))
        ln = 6000 if rng.random() < 0.5 else int(rng.integers(300, 6001))
        seg = fam[f, 6000 - ln:].copy()
        substitute(seg, np.flatnonzero(rng.random(ln) < 0.05), rng)
        dst = int(rng.integers(0, n - ln))
        _plant(g, seg, dst, rng.integers(0, 2))
        regions.append((dst, dst + ln, "fam6k"))
        done += ln
    # tandem arrays
    total = int(0.05 * n)
    done = 0
    while done < total:
        u = int(rng.integers(2, 51))
        ln = int(rng.integers(100, 20_001))
        arr = np.resize(rng.integers(0, 4, size=u, dtype=np.uint8), ln)
        substitute(arr, np.flatnonzero(rng.random(ln) < rng.uniform(0.01, 0.05)), rng)
        dst = int(rng.integers(0, n - ln))
        g[dst:dst + ln] = arr
        regions.append((dst, dst + ln, "tandem"))
        done += ln
    return Genome(g, regions)


def donor_of(genome: Genome, seed: int = SEED_DONOR_HUMAN, snv_rate: float = 0.001) -> np.ndarray:
    """The sequenced individual: the reference with i.i.d. single-base
    substitutions at `snv_rate` (no indels: the search is substitution-only)."""
    rng = _rng(seed)
    d = genome.codes.copy()
    where = np.unique(rng.integers(0, genome.n, size=int(snv_rate * genome.n)))
    substitute(d, where, rng)
    return d


def paired_reads(donor: np.ndarray, n_pairs: int, seed: int = SEED_READS_HUMAN, m: int = 150,
                 insert_mean: float = 500.0, insert_sd: float = 50.0, err: float = 0.01,
                 chunk: int = 500_000) -> ReadBatch:
    """Paired-end reads, mates interleaved (read 2i = mate 1, 2i + 1 = mate 2).

    Fragment length round(Normal(500, 50)) clipped to [300, 700], start
    uniform; on a + fragment mate 1 is its first m bases and mate 2 the
    reverse complement of its last m bases; a - fragment swaps the roles.
    Each base then carries an i.i.d. sequencing substitution with
    probability `err`.  origin/strand record each mate's true placement on
    the reference coordinates (the donor has the same coordinates).
    """
    rng = _rng(seed)
    N = len(donor)
    n = 2 * n_pairs
    nw = (m + 15) // 16
    off = (np.arange(n + 1, dtype=np.uint64) * nw).astype(np.uint64)
    words = np.zeros(n * nw, dtype=np.uint32)
    origin = np.zeros(n, dtype=np.int64)
    strand = np.zeros(n, dtype=np.uint8)
    n_subs = np.zeros(n, dtype=np.int32)
    for p0 in range(0, n_pairs, chunk):
        c = min(chunk, n_pairs - p0)
        L = np.clip(np.rint(rng.normal(insert_mean, insert_sd, size=c)), 300, 700).astype(np.int64)
        s = (rng.random(c) * (N - L + 1)).astype(np.int64)
        fwd = rng.integers(0, 2, size=c) == 0
        left = donor[s[:, None] + np.arange(m)[None, :]]
        right = donor[(s + L - m)[:, None] + np.arange(m)[None, :]]
        right_rc = (3 - right)[:, ::-1]
        left_rc = (3 - left)[:, ::-1]
        m1 = np.where(fwd[:, None], left, right_rc)
        m2 = np.where(fwd[:, None], right_rc, left)
        mates = np.empty((2 * c, m), dtype=np.uint8)
        mates[0::2] = m1
        mates[1::2] = m2
        hit = rng.random(mates.shape) < err
        shift = rng.integers(1, 4, size=mates.shape, dtype=np.uint8)
        mates = np.where(hit, (mates + shift) & 3, mates).astype(np.uint32)
        r0 = 2 * p0
        idx = np.arange(r0, r0 + 2 * c)
        _pack_group(words, off, idx, mates)
        o = np.empty(2 * c, dtype=np.int64)
        o[0::2] = np.where(fwd, s, s + L - m)
        o[1::2] = np.where(fwd, s + L - m, s)
        st = np.empty(2 * c, dtype=np.uint8)
        st[0::2] = np.where(fwd, 0, 1)
        st[1::2] = np.where(fwd, 1, 0)
        origin[r0:r0 + 2 * c] = o
        strand[r0:r0 + 2 * c] = st
        n_subs[r0:r0 + 2 * c] = hit.sum(axis=1)
    return ReadBatch(words, off, np.full(n, m, dtype=np.uint16), np.full(n, 2, dtype=np.uint8),
                     origin, strand, n_subs)


def serve_requests(donor: np.ndarray, n_requests: int, seed: int = SEED_READS_SERVE,
                   size_range=(1_000, 1_000_000), max_size: int | None = None) -> list:
    """Serving requests: sizes log-uniform in `size_range` (clipped to
    `max_size` when given); every read's length uniform over {100, 150, 250}
    bp and its k uniform in {0, 1, 2}; reads drawn from the donor as the
    human-scale mates are (uniform origin, fair strand, 1% i.i.d.
    substitutions)."""
    rng = _rng(seed)
    lo, hi = size_range
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_requests)).astype(np.int64)
    if max_size is not None:
        sizes = np.minimum(sizes, max_size)
    g = Genome(donor)
    out = []
    for s in sizes:
        lengths = rng.choice(np.array([100, 150, 250]), size=int(s))
        k = rng.integers(0, 3, size=int(s)).astype(np.uint8)
        out.append(sample_reads(g, lengths, k, rng, subs="rate", sub_rate=0.01))
    return out


# --------------------------------------------------------------------------
# A reference of several contigs, as FASTA files hold them
# --------------------------------------------------------------------------

IUPAC_AMBIGUOUS = b"NRYKMSWBDHV"


def multi_contig_reference(lengths=(3000, 1700, 2600, 900), seed: int = SEED_REFERENCE, *,
                           shared: int = 400) -> list:
    """Contig byte strings with what real references hold besides A/C/G/T:
    lower-case stretches (soft-masked repeats, 5% of bases in runs of up to
    200), runs of N (assembly gaps: two per contig, 1-60 bases), scattered
    single IUPAC ambiguity codes (0.2% of bases), and a ``shared``-base
    segment of contig 0 copied into contig 2 and, reverse-complemented and
    with one substitution per 50 bases, into contig 3 (so that reads land on
    several contigs, on both strands, at several substitution counts)."""
    rng = _rng(seed)
    codes = [rng.integers(0, 4, size=n, dtype=np.uint8) for n in lengths]
    if len(codes) >= 4 and shared and min(lengths[0], lengths[2], lengths[3]) > shared + 200:
        seg = codes[0][100:100 + shared].copy()
        codes[2][150:150 + shared] = seg
        codes[3][50:50 + shared] = opposite_strand(seg)
        substitute(codes[3], 50 + np.arange(25, shared, 50), rng)   # a near copy: one change per 50 bases
    out = []
    for c in codes:
        b = bytearray(ACGT[c].tobytes())
        n = len(b)
        for _ in range(max(1, n // 4000)):      # soft-masked stretches
            a = int(rng.integers(0, n))
            for j in range(a, min(n, a + int(rng.integers(1, 201)))):
                b[j] |= 0x20
        for _ in range(2):                      # N gaps
            ln = int(rng.integers(1, 61))
            a = int(rng.integers(0, max(1, n - ln)))
            b[a:a + ln] = b"N" * ln
        for j in np.flatnonzero(rng.random(n) < 0.002):   # single ambiguity codes
            b[int(j)] = IUPAC_AMBIGUOUS[int(rng.integers(0, len(IUPAC_AMBIGUOUS)))]
        out.append(bytes(b))
    return out


def to_fasta(contigs, names, width: int = 60, crlf: bool = False) -> bytes:
    """FASTA text of the contigs, sequence lines of ``width`` bytes."""
    nl = b"\r\n" if crlf else b"\n"
    parts = []
    for name, seq in zip(names, contigs):
        parts.append(b">" + name.encode() + b" synthetic contig" + nl)
        for a in range(0, len(seq), width):
            parts.append(seq[a:a + width] + nl)
    return b"".join(parts)


# --------------------------------------------------------------------------
# Reads as FASTQ text
# --------------------------------------------------------------------------

SEED_FASTQ = 71


def to_fastq(batch: ReadBatch, *, n_frac: float = 0.3, max_n: int = 3, lower_frac: float = 0.1,
             mate_suffix: bool = False, crlf: bool = False, seed: int = SEED_FASTQ) -> tuple:
    """FASTQ text of a batch as a sequencer writes it: names with a comment
    after a space, qualities in '!'..'J', a fraction ``n_frac`` of reads with
    1..``max_n`` bases turned into N (or another IUPAC code), and a fraction
    ``lower_frac`` of reads in lower case.  With ``mate_suffix``, reads 2i and
    2i + 1 are written to two texts as "/1" and "/2" mates of one name.
    Returns (texts, ambiguous offsets per read, qualities per read)."""
    rng = _rng(seed)
    nl = b"\r\n" if crlf else b"\n"
    texts = [[], []] if mate_suffix else [[]]
    amb, quals = [], []
    for i in range(batch.n):
        seq = bytearray(ACGT[batch.read(i)].tobytes())
        m = len(seq)
        pos = []
        if rng.random() < n_frac:
            pos = sorted(rng.choice(m, size=int(rng.integers(1, max_n + 1)), replace=False).tolist())
            for j in pos:
                seq[j] = IUPAC_AMBIGUOUS[int(rng.integers(0, len(IUPAC_AMBIGUOUS)))] if rng.random() < 0.2 else ord("N")
        if rng.random() < lower_frac:
            seq = bytearray(bytes(seq).lower())
        q = bytes(rng.integers(33, 75, size=m, dtype=np.uint8))
        amb.append(pos)
        quals.append(q.decode())
        if mate_suffix:
            name = f"frag{i // 2}/{i % 2 + 1}".encode()
            out = texts[i % 2]
        else:
            name = f"read{i}".encode()
            out = texts[0]
        out.append(b"@" + name + b" lane=1" + nl + bytes(seq) + nl + b"+" + nl + q + nl)
    return [b"".join(t) for t in texts], amb, quals
