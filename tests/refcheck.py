"""Independent brute-force helpers used by the tests to pin the oracle.

Pure numpy / Python written from the definitions only (no FM index): the
suffix array as sorted suffixes, occurrence counts by sliding windows, and the
Hamming-distance hit set of Section 2's "align with few mismatches" step.
"""
from __future__ import annotations

import numpy as np


def rc(codes: np.ndarray) -> np.ndarray:
    return (3 - np.asarray(codes, dtype=np.int16))[::-1].astype(np.uint8)


def suffix_array_by_definition(g: np.ndarray) -> np.ndarray:
    """Sort the suffixes of G$ as Python tuples ($ = -1 is smallest)."""
    t = [int(x) for x in g] + [-1]
    return np.array(sorted(range(len(t)), key=lambda i: t[i:]), dtype=np.uint32)


def windows(g: np.ndarray, m: int) -> np.ndarray:
    return np.lib.stride_tricks.sliding_window_view(np.asarray(g, dtype=np.uint8), m)


def count_occurrences(g: np.ndarray, p: np.ndarray) -> int:
    if len(p) > len(g):
        return 0
    return int(np.all(windows(g, len(p)) == p[None, :], axis=1).sum())


def hamming_hits(g: np.ndarray, read: np.ndarray, k: int) -> list:
    """Sorted [(pos, strand, d)] with d = Ham(R or rc(R), G[p, p+m)) <= k."""
    m = len(read)
    if m > len(g):
        return []
    w = windows(g, m)
    out = []
    for strand, p in ((0, read), (1, rc(read))):
        d = (w != p[None, :]).sum(axis=1)
        for pos in np.flatnonzero(d <= k):
            out.append((int(pos), strand, int(d[pos])))
    return sorted(out)


def lower_bound_breakpoints(g: np.ndarray, pattern: np.ndarray, k: int, q: int) -> list:
    """The mismatch lower bound of the pruned search, from its definition:
    scan P[0, m - q') left to right (q' = min(m, q)), cutting it into maximal
    pieces that occur in G; each piece P[s, j] that does not occur ends at j
    (the next starts at j + 1) and gives the breakpoint j + 1.  Stops after
    k + 1 breakpoints.  Substring occurrence is plain `bytes in bytes`."""
    text = np.asarray(g, dtype=np.uint8).tobytes()
    p = np.asarray(pattern, dtype=np.uint8)
    lim = len(p) - min(len(p), q)
    out, s = [], 0
    for j in range(lim):
        if p[s:j + 1].tobytes() not in text:
            out.append(j + 1)
            s = j + 1
            if len(out) > k:
                break
    return out


def lb_word(breakpoints: list) -> int:
    """Pack breakpoints as the GPU does: 9-bit field t = t-th breakpoint, 511 unused."""
    v = (1 << 64) - 1
    for t, b in enumerate(breakpoints):
        v &= ~(511 << (9 * t))
        v |= b << (9 * t)
    return v


def min_prefix_mismatches(g: np.ndarray, pattern: np.ndarray, i: int) -> int:
    """min over placements of Ham(P[0, i), G[p, p+i)) by brute force (0 for i = 0)."""
    if i == 0:
        return 0
    w = windows(g, i)
    return int((w != np.asarray(pattern[:i], dtype=np.uint8)[None, :]).sum(axis=1).min())


def contig_hamming_hits(contigs, read: np.ndarray, k: int) -> list:
    """Sorted [(pos, strand, d)] over a reference of several contigs, from the
    definition on each contig's own bytes: a window counts only when it lies
    inside one contig and holds no byte other than A/C/G/T (either case);
    pos is the window's start in the contigs laid back to back."""
    value = np.full(256, 255, dtype=np.uint8)
    for ch, v in zip(b"ACGT", range(4)):
        value[ch] = v
        value[ch + 32] = v
    out, base = [], 0
    for seq in contigs:
        c = value[np.frombuffer(bytes(seq), dtype=np.uint8)]
        for pos, strand, d in hamming_hits(np.where(c == 255, 0, c), read, k):
            if not np.any(c[pos:pos + len(read)] == 255):
                out.append((base + pos, strand, d))
        base += len(seq)
    return sorted(out)


def hamming_hits_n(g: np.ndarray, read: np.ndarray, k: int) -> list:
    """Sorted [(pos, strand, d)] for a read whose ambiguous bases are coded
    255: such a base equals no genome base on either strand."""
    p = np.asarray(read, dtype=np.int16)
    rcp = np.where(p == 255, 255, 3 - p)[::-1]
    m = len(p)
    if m > len(g):
        return []
    w = windows(g, m).astype(np.int16)
    out = []
    for strand, q in ((0, p), (1, rcp)):
        d = (w != q[None, :]).sum(axis=1)
        for pos in np.flatnonzero(d <= k):
            out.append((int(pos), strand, int(d[pos])))
    return sorted(out)
