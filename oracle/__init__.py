"""CPU oracle for the k-mismatch FM-index read search (MICA, Section 2).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark are the only callers.  The product path (the CUDA library
and its binding) never imports this package, and this package never imports
the product.  The arithmetic lives in ``oracle.c`` (plain C, compiled with
gcc by :func:`build`); this module only marshals numpy arrays.

Functions and what pins them (tests/test_oracle_*.py):

* :func:`sa_sort`, :func:`sa_is` -- suffix array of T = G$ by sorting and by
  SA-IS; pinned against Python's ``sorted`` of the suffixes (the definition)
  and against each other on random and periodic strings.
* :class:`FMIndex` (BWT, C, Occ) -- pinned by LF consistency
  (SA[LF(j)] = SA[j]-1), the column sums of Occ, and exact-pattern interval
  sizes equal to brute-force occurrence counts.
* :func:`align` -- pinned against a brute-force Hamming scan written in
  numpy inside the tests, the generator's ground truth on the 1 Mbp random
  genome (chance hits are vanishingly rare there), reverse-complement symmetry,
  and for the hit cap by the properties that define it.
* :func:`bruteforce` -- pinned against the numpy scan in the tests.
* :func:`reference_concat`, :func:`reference_filter` -- references of
  several contigs with ambiguous bases: the concatenated text and the rule
  that keeps a hit only when its window lies in one contig and covers no
  ambiguous byte.  :func:`splitmix64` is pinned by the published outputs of
  its reference implementation (tests/golden/splitmix64.txt); the filtered
  search is pinned by a brute-force Hamming scan of each contig's own bytes
  that skips windows with ambiguous bytes (tests/test_reference.py).
* :func:`n_filter` -- reads with ambiguous bases (N): each such base costs
  one substitution wherever it falls; pinned by a brute-force Hamming scan
  in which the read's ambiguous bases equal no base (tests/test_fastq.py).
* :func:`pair` -- mate pairing of a result (the paper's properly paired
  reads, Section 3, Table 1), plain Python loops over every combination of
  listed hits; pinned by the generator's true fragments on a random genome
  (every pair found concordant at its true fragment, with its true
  substitutions) and by hand-worked cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

HIT_DTYPE = np.dtype([("pos", "<u4"), ("strand", "u1"), ("mm", "u1"), ("pad", "<u2")])


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    sig = {
        "oracle_sa_sort": (i32, [P, u64, P]),
        "oracle_sa_is": (i32, [P, u64, P]),
        "oracle_fm_new": (P, [P, u64, i32, P]),
        "oracle_fm_free": (None, [P]),
        "oracle_occ": (u64, [P, i32, u64]),
        "oracle_C": (u64, [P, i32]),
        "oracle_rows": (u64, [P]),
        "oracle_copy_sa": (None, [P, P]),
        "oracle_copy_bwt": (None, [P, P]),
        "oracle_exact_interval": (None, [P, P, u32, P, P]),
        "oracle_align": (P, [P, P, P, P, P, u64, u32, i32]),
        "oracle_bruteforce": (P, [P, u64, P, P, P, P, u64, i32]),
        "oracle_result_free": (None, [P]),
        "oracle_result_n": (u64, [P]),
        "oracle_result_status": (i32, [P]),
        "oracle_result_nodes": (u64, [P]),
        "oracle_result_copy": (None, [P, P, P, P]),
        "oracle_result_n_hits": (u64, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _codes(g) -> np.ndarray:
    g = np.ascontiguousarray(g, dtype=np.uint8)
    if g.size and g.max() > 3:
        raise ValueError("genome codes must be 0..3")
    return g


def sa_sort(g) -> np.ndarray:
    """Suffix array of G$ by sorting the suffixes (small inputs)."""
    g = _codes(g)
    sa = np.empty(len(g) + 1, dtype=np.uint32)
    if _load().oracle_sa_sort(_ptr(g), len(g), _ptr(sa)):
        raise MemoryError("oracle_sa_sort")
    return sa


def sa_is(g) -> np.ndarray:
    """Suffix array of G$ by SA-IS."""
    g = _codes(g)
    sa = np.empty(len(g) + 1, dtype=np.uint32)
    if _load().oracle_sa_is(_ptr(g), len(g), _ptr(sa)):
        raise MemoryError("oracle_sa_is")
    return sa


class Result:
    """Per-read hit lists in CSR form: ``hits[offsets[i]:offsets[i+1]]``."""

    def __init__(self, total, offsets, hits, nodes=0):
        self.total = total
        self.offsets = offsets
        self.hits = hits
        self.nodes = nodes

    def read_hits(self, i: int) -> np.ndarray:
        return self.hits[int(self.offsets[i]):int(self.offsets[i + 1])]

    def as_tuples(self, i: int) -> list:
        h = self.read_hits(i)
        return [(int(p), int(s), int(d)) for p, s, d in zip(h["pos"], h["strand"], h["mm"])]


def _take_result(lib, handle) -> Result:
    if not handle:
        raise ValueError("oracle rejected the input (k > 3, empty read or read longer than genome)")
    try:
        if lib.oracle_result_status(handle) != 0:
            raise MemoryError("oracle out of memory")
        n = lib.oracle_result_n(handle)
        total = np.empty(n, dtype=np.uint64)
        offsets = np.empty(n + 1, dtype=np.uint64)
        hits = np.empty(max(1, lib.oracle_result_n_hits(handle)), dtype=HIT_DTYPE)
        lib.oracle_result_copy(handle, _ptr(total), _ptr(offsets), _ptr(hits))
        hits = hits[:int(offsets[-1])].copy()
        return Result(total, offsets, hits, int(lib.oracle_result_nodes(handle)))
    finally:
        lib.oracle_result_free(handle)


class FMIndex:
    """Plain FM index of G$ with the full suffix array (oracle side)."""

    def __init__(self, g, sa_method: str = "auto", sa=None):
        lib = _load()
        self.g = _codes(g)
        self.n = len(self.g)
        if sa is not None:
            sa = np.ascontiguousarray(sa, dtype=np.uint32)
            meth, sap = 0, _ptr(sa)
        else:
            if sa_method == "auto":
                sa_method = "sort" if self.n <= 200_000 else "sais"
            meth, sap = (0 if sa_method == "sort" else 1), None
        self._h = lib.oracle_fm_new(_ptr(self.g), self.n, meth, sap)
        if not self._h:
            raise MemoryError("oracle_fm_new")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.oracle_fm_free(h)
            self._h = None

    @property
    def rows(self) -> int:
        return self.n + 1

    def C(self, c: int) -> int:
        return int(_lib.oracle_C(self._h, c))

    def occ(self, c: int, i: int) -> int:
        return int(_lib.oracle_occ(self._h, c, i))

    def sa(self) -> np.ndarray:
        out = np.empty(self.rows, dtype=np.uint32)
        _lib.oracle_copy_sa(self._h, _ptr(out))
        return out

    def bwt(self) -> np.ndarray:
        """BWT symbols: 0..3 = A..T, 4 = $."""
        out = np.empty(self.rows, dtype=np.uint8)
        _lib.oracle_copy_bwt(self._h, _ptr(out))
        return out

    def exact_interval(self, p) -> tuple:
        p = np.ascontiguousarray(p, dtype=np.uint8)
        l, r = ctypes.c_uint64(), ctypes.c_uint64()
        _lib.oracle_exact_interval(self._h, _ptr(p), len(p), ctypes.byref(l), ctypes.byref(r))
        return int(l.value), int(r.value)

    def align(self, batch, cap: int = 0, threads: int = 0) -> Result:
        """All hits of every read of ``batch`` (a synth.ReadBatch or any object
        with words/word_off/lengths/k arrays), both strands, <= k mismatches."""
        words, off, lens, k = _batch_arrays(batch)
        h = _lib.oracle_align(self._h, _ptr(words), _ptr(off), _ptr(lens), _ptr(k),
                              len(lens), cap, threads)
        return _take_result(_lib, h)

    def align_best_stratum(self, batch, cap: int = 0, threads: int = 0) -> Result:
        """Best-stratum reporting: of each read's hits (all of them, from
        :meth:`align` without a cap) only those with the read's smallest d;
        total = their number; over the cap, the first `cap` in the order
        (strand, SA row of the window's position), listed by (pos, strand, d)."""
        full = self.align(batch, cap=0, threads=threads)
        sa = self.sa().astype(np.int64)
        isa = np.empty_like(sa)
        isa[sa] = np.arange(sa.size)
        n = len(full.total)
        total = np.zeros(n, dtype=np.uint64)
        lists = []
        for i in range(n):
            h = full.as_tuples(i)
            if h:
                dmin = min(d for _, _, d in h)
                h = [x for x in h if x[2] == dmin]
            total[i] = len(h)
            if cap and len(h) > cap:
                h = sorted(sorted(h, key=lambda x: (x[1], int(isa[x[0]])))[:cap])
            lists.append(h)
        offsets = np.zeros(n + 1, dtype=np.uint64)
        offsets[1:] = np.cumsum([len(x) for x in lists])
        hits = np.zeros(int(offsets[-1]), dtype=HIT_DTYPE)
        j = 0
        for h in lists:
            for (p, st, d) in h:
                hits[j] = (p, st, d, 0)
                j += 1
        return Result(total, offsets, hits, full.nodes)


def _batch_arrays(batch):
    words = np.ascontiguousarray(batch.words, dtype=np.uint32)
    if words.size == 0:
        words = np.zeros(1, dtype=np.uint32)
    off = np.ascontiguousarray(batch.word_off, dtype=np.uint64)
    lens = np.ascontiguousarray(batch.lengths, dtype=np.uint16)
    k = np.ascontiguousarray(batch.k, dtype=np.uint8)
    return words, off, lens, k


def bruteforce(g, batch, threads: int = 0) -> Result:
    """Hamming scan of every window of both strands (tiny inputs only)."""
    lib = _load()
    g = _codes(g)
    words, off, lens, k = _batch_arrays(batch)
    h = lib.oracle_bruteforce(_ptr(g), len(g), _ptr(words), _ptr(off), _ptr(lens), _ptr(k),
                              len(lens), threads)
    return _take_result(lib, h)


def pair(result: Result, lengths, insert_min: int, insert_max: int) -> list:
    """For each pair i (reads 2i, 2i+1): every listed + strand hit a of one
    mate with every listed - strand hit b of the other, concordant when
    L = b.pos + m_b - a.pos is in [insert_min, insert_max] (m_b: the length
    of b's read).  Returns per pair (n_concordant, n_best, pos_plus,
    pos_minus, plus_mate, mm): the count, the smallest a.mm + b.mm, how many
    combinations reach it, and the best one by (mm, pos_plus, plus_mate,
    pos_minus); zeros when there is none."""
    lengths = np.asarray(lengths)
    out = []
    for p in range((len(result.offsets) - 1) // 2):
        mates = [result.as_tuples(2 * p), result.as_tuples(2 * p + 1)]
        combos = []
        for amate in (0, 1):
            bmate = 1 - amate
            mb = int(lengths[2 * p + bmate])
            for (apos, astr, ad) in mates[amate]:
                if astr != 0:
                    continue
                for (bpos, bstr, bd) in mates[bmate]:
                    if bstr != 1:
                        continue
                    frag = bpos + mb - apos
                    if insert_min <= frag <= insert_max:
                        combos.append((ad + bd, apos, amate, bpos))
        if not combos:
            out.append((0, 0, 0, 0, 0, 0))
            continue
        best = min(combos)
        n_best = sum(1 for c in combos if c[0] == best[0])
        out.append((len(combos), n_best, best[1], best[3], best[2], best[0]))
    return out



# --------------------------------------------------------------------------
# References of several contigs with ambiguous bases
# --------------------------------------------------------------------------

_M64 = (1 << 64) - 1


def splitmix64(state: int) -> int:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output when the
    generator's state before the call is ``state``."""
    z = (state + 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def reference_concat(contigs) -> tuple:
    """The text G of a reference given as a list of contig byte strings (any
    case; a byte other than A/C/G/T is ambiguous): the contigs back to back,
    each ambiguous byte at coordinate j replaced by base splitmix64(j) >> 62.
    Returns (codes uint8[N], starts [n + 1 contig bounds], runs [(s, e)]
    maximal runs of ambiguous coordinates).  Plain loops; small inputs."""
    codes, starts, runs = [], [0], []
    value = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}
    for seq in contigs:
        for byte in bytes(seq).upper():
            j = len(codes)
            if byte in value:
                codes.append(value[byte])
                continue
            codes.append(splitmix64(j) >> 62)
            if runs and runs[-1][1] == j:
                runs[-1] = (runs[-1][0], j + 1)
            else:
                runs.append((j, j + 1))
        starts.append(len(codes))
    return np.array(codes, dtype=np.uint8), starts, runs


def on_reference(pos: int, m: int, starts, runs) -> bool:
    """Whether the window [pos, pos + m) of G lies inside one contig and
    covers no ambiguous coordinate (a placement on the reference)."""
    inside = any(starts[c] <= pos and pos + m <= starts[c + 1] for c in range(len(starts) - 1))
    clear = not any(s < pos + m and pos < e for s, e in runs)
    return inside and clear


def reference_filter(result: Result, lengths, starts, runs) -> tuple:
    """Drop the listed hits that are not placements on the reference; each
    read's total falls by the number dropped from its list.  Returns
    (Result, number dropped)."""
    lengths = np.asarray(lengths)
    n = len(result.offsets) - 1
    total = np.array(result.total, dtype=np.uint64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    kept, dropped = [], 0
    for i in range(n):
        m = int(lengths[i])
        for h in result.read_hits(i):
            if on_reference(int(h["pos"]), m, starts, runs):
                kept.append(h)
            else:
                total[i] -= 1
                dropped += 1
        offsets[i + 1] = len(kept)
    hits = np.array(kept, dtype=HIT_DTYPE) if kept else np.zeros(0, dtype=HIT_DTYPE)
    return Result(total, offsets, hits), dropped


# --------------------------------------------------------------------------
# Reads with ambiguous bases
# --------------------------------------------------------------------------

def n_filter(result: Result, reads, ambiguous, k, g) -> tuple:
    """Ambiguous read bases count as substitutions wherever they fall.

    reads[i]: read i's base codes as searched (ambiguous offsets hold some
    stand-in base); ambiguous[i]: its ambiguous offsets; k[i]: its budget;
    g: the text's base codes.  For every read with ambiguous bases, each
    listed hit's d becomes d' = the window offsets whose reference base
    differs from the read's base or whose read base is ambiguous (the read
    reverse-complemented on the - strand), and hits with d' > k[i] are
    dropped, total falling by their number.  Returns (Result, dropped)."""
    g = np.asarray(g)
    n = len(result.offsets) - 1
    total = np.array(result.total, dtype=np.uint64)
    offsets = np.zeros(n + 1, dtype=np.uint64)
    kept, dropped = [], 0
    for i in range(n):
        amb = set(int(j) for j in ambiguous[i])
        read = [int(c) for c in reads[i]]
        m = len(read)
        for h in result.read_hits(i):
            if not amb:
                kept.append(h)
                continue
            pos, strand = int(h["pos"]), int(h["strand"])
            d = 0
            for j in range(m):
                r = m - 1 - j if strand else j            # read offset at window offset j
                base = 3 - read[r] if strand else read[r]
                if r in amb or int(g[pos + j]) != base:
                    d += 1
            if d <= int(k[i]):
                kept.append((pos, strand, d, 0))
            else:
                total[i] -= 1
                dropped += 1
        offsets[i + 1] = len(kept)
    hits = np.array(kept, dtype=HIT_DTYPE) if kept else np.zeros(0, dtype=HIT_DTYPE)
    return Result(total, offsets, hits), dropped
