"""A second, plain-Python statement of the SAM records the library writes for
a search result against a reference of several contigs (test side only).

Rules (SAM 1.6 for the fields; the library's readings for what SAM leaves
open): per read, V = its listed hits whose window lies inside one contig and
covers no ambiguous byte; the primary is the first hit of V with the fewest
substitutions; SEQ is stored on the forward strand; CIGAR mM; NM/MD against
the reference text; X0/X1 = hits of V at the best stratum and the next one;
ZT = total less the listed hits dropped; MAPQ 0 / 25 / 37 by uniqueness;
pairs take the best concordant placement of the pairing when both its hits
are in V and in one contig (properly paired), else each mate its own primary.
"""
from __future__ import annotations

import numpy as np

import oracle

ACGT = "ACGT"


def _codes(batch, i: int) -> list:
    m = int(batch.lengths[i])
    w = batch.words[int(batch.word_off[i]):int(batch.word_off[i + 1])]
    return [int((int(w[j // 16]) >> (2 * (j % 16))) & 3) for j in range(m)]


def _oriented(codes: list, strand: int) -> list:
    return codes if strand == 0 else [3 - c for c in reversed(codes)]


class _Read:
    """rec = (name, qualities, ambiguous offsets, k) for a read from FASTQ."""

    def __init__(self, batch, result, i, starts, runs, text, rec=None):
        self.codes = _codes(batch, i)
        self.m = len(self.codes)
        self.name, self.qual = (rec[0], rec[1]) if rec else (None, None)
        self.amb = set(rec[2]) if rec else set()
        kmax = rec[3] if rec else 3
        listed = result.as_tuples(i)
        total = int(result.total[i])
        self.V = []
        raws = []
        for pos, strand, mm in listed:
            raw, d = mm, mm
            if self.amb:
                ori = _oriented(self.codes, strand)
                offs = [self.m - 1 - j if strand else j for j in range(self.m)]
                raw = sum(1 for j in range(self.m) if text[pos + j] != ACGT[ori[j]])
                d = sum(1 for j in range(self.m) if text[pos + j] != ACGT[ori[j]] or offs[j] in self.amb)
            raws.append(raw)
            if oracle.on_reference(pos, self.m, starts, runs) and d <= kmax:
                c = max(j for j in range(len(starts) - 1) if starts[j] <= pos)
                self.V.append((pos, strand, d, c, pos - starts[c]))
        self.primary = None
        self.c0 = self.c1 = 0
        self.mapq = 0
        self.complete = total == len(listed)
        self.zt = total - (len(listed) - len(self.V))
        if not self.V:
            return
        dmin = min(v[2] for v in self.V)
        self.primary = next(v for v in self.V if v[2] == dmin)
        self.c0 = sum(1 for v in self.V if v[2] == dmin)
        self.c1 = sum(1 for v in self.V if v[2] == dmin + 1)
        # the cap cut the search's highest d first
        unique = self.c0 == 1 and (self.complete or any(r > dmin for r in raws))
        if unique:
            sure = self.c1 == 0 and (self.complete or any(r > dmin + 1 for r in raws))
            self.mapq = 37 if sure else 25

    def seq(self, strand):
        s = "".join("N" if (self.m - 1 - j if strand else j) in self.amb else ACGT[c]
                    for j, c in enumerate(_oriented(self.codes, strand)))
        q = "*" if self.qual is None else (self.qual[::-1] if strand else self.qual)
        return s, q


def _md(seq: str, window: str) -> str:
    out, run = [], 0
    for c, g in zip(seq, window):
        if c == g:
            run += 1
        else:
            out.append(f"{run}{g}")
            run = 0
    return "".join(out) + str(run)


def sam_text(names, starts, runs, text: str, batch, result, pairs=None, prefix: str = "r",
             secondary: bool = False, command_line: str | None = None, first_id: int = 0,
             records=None) -> str:
    """The whole SAM file (header and records) as a string; records: per
    read (name, qualities, ambiguous offsets, k) for a batch from FASTQ."""
    lines = ["@HD\tVN:1.6\tSO:unsorted"]
    for j, name in enumerate(names):
        lines.append(f"@SQ\tSN:{name}\tLN:{starts[j + 1] - starts[j]}")
    pg = "@PG\tID:mica-gb300\tPN:mica-gb300\tVN:1.0"
    lines.append(pg + (f"\tCL:{command_line}" if command_line else ""))
    n = len(batch.lengths)
    reads = [_Read(batch, result, i, starts, runs, text, records[i] if records else None) for i in range(n)]

    def match_tags(r, v):
        pos, strand, d = v[0], v[1], v[2]
        return [f"NM:i:{d}", "MD:Z:" + _md(r.seq(strand)[0], text[pos:pos + r.m])]

    def record(qname, flag, r, v, mapq, here, mate, tlen):
        # here / mate: (contig, pos1) or None
        rname = names[here[0]] if here else "*"
        pos1 = here[1] if here else 0
        if mate is None:
            rnext, pnext = "*", 0
        else:
            rnext, pnext = ("=" if here and mate[0] == here[0] else names[mate[0]]), mate[1]
        if r.name is not None:
            qname = r.name
        if v is None:
            fields = [qname, flag | 4, rname, pos1, 0, "*", rnext, pnext, tlen, *r.seq(0)]
            return "\t".join(map(str, fields))
        flag |= 16 if v[1] else 0
        fields = [qname, flag, rname, pos1, mapq, f"{r.m}M", rnext, pnext, tlen, *r.seq(v[1])]
        fields += match_tags(r, v) + [f"X0:i:{r.c0}", f"X1:i:{r.c1}", f"ZT:i:{r.zt}"]
        return "\t".join(map(str, fields))

    def secondaries(qname, flag, r, v, mate):
        if not secondary:
            return []
        out = []
        for s in r.V:
            if s is v:
                continue
            here = (s[3], s[4] + 1)
            if mate is None:
                rnext, pnext = "*", 0
            else:
                rnext, pnext = ("=" if mate[0] == here[0] else names[mate[0]]), mate[1]
            f = flag | 256 | (16 if s[1] else 0)
            q = r.name if r.name is not None else qname
            fields = [q, f, names[s[3]], s[4] + 1, 0, f"{r.m}M", rnext, pnext, 0, "*", "*"]
            out.append("\t".join(map(str, fields + match_tags(r, s))))
        return out

    if pairs is None:
        for i, r in enumerate(reads):
            q = f"{prefix}{first_id + i}"
            here = (r.primary[3], r.primary[4] + 1) if r.primary else None
            lines.append(record(q, 0, r, r.primary, r.mapq, here, None, 0))
            lines += secondaries(q, 0, r, r.primary, None)
        return "\n".join(lines) + "\n"

    for p in range(n // 2):
        r1, r2 = reads[2 * p], reads[2 * p + 1]
        row = pairs[p]
        n_conc, n_best = int(row["n_concordant"]), int(row["n_best"])
        pos_plus, pos_minus, plus_mate = int(row["pos_plus"]), int(row["pos_minus"]), int(row["plus_mate"])
        p1, p2, q1, q2, proper = r1.primary, r2.primary, r1.mapq, r2.mapq, False
        if n_conc:
            plus, minus = (r1, r2) if plus_mate == 0 else (r2, r1)
            a = next((v for v in plus.V if v[0] == pos_plus and v[1] == 0), None)
            b = next((v for v in minus.V if v[0] == pos_minus and v[1] == 1), None)
            if a is not None and b is not None and a[3] == b[3]:
                p1, p2 = (a, b) if plus_mate == 0 else (b, a)
                q = 0 if n_best > 1 else (37 if n_conc == 1 and r1.complete and r2.complete else 25)
                q1 = q2 = q
                proper = True
        h1 = (p1[3], p1[4] + 1) if p1 else None
        h2 = (p2[3], p2[4] + 1) if p2 else None
        if p1 is None:
            h1 = h2
        if p2 is None:
            h2 = h1
        t1 = t2 = 0
        if p1 and p2 and p1[3] == p2[3]:
            lo = min(p1[4], p2[4])
            hi = max(p1[4] + r1.m, p2[4] + r2.m)
            t = hi - lo
            first1 = p1[4] < p2[4] or (p1[4] == p2[4])
            t1, t2 = (t, -t) if first1 else (-t, t)
        base = 1 | (2 if proper else 0)
        f1 = base | 64 | ((32 if p2[1] else 0) if p2 else 8)
        f2 = base | 128 | ((32 if p1[1] else 0) if p1 else 8)
        q = f"{prefix}{first_id + p}"
        lines.append(record(q, f1, r1, p1, q1, h1, h2, t1))
        lines += secondaries(q, f1 & ~2, r1, p1, h2)
        lines.append(record(q, f2, r2, p2, q2, h2, h1, t2))
        lines += secondaries(q, f2 & ~2, r2, p2, h1)
    return "\n".join(lines) + "\n"


def pairs_array(tuples, dtype) -> np.ndarray:
    """oracle.pair tuples -> rows of the library's pairing record."""
    out = np.zeros(len(tuples), dtype=dtype)
    for i, (nc, nb, pp, pm, mate, mm) in enumerate(tuples):
        out[i] = (nc, nb, pp, pm, mate, mm, 0)
    return out


def no_pairs(n_pairs: int, dtype) -> np.ndarray:
    """Pairing rows with no concordant placement (mates written as pairs)."""
    return np.zeros(n_pairs, dtype=dtype)
