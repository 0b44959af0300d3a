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
