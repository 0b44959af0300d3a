"""Reader for tests/golden/handworked_hits.txt (hand-worked hit sets)."""
import os

import numpy as np

import synth

_PATH = os.path.join(os.path.dirname(__file__), "golden", "handworked_hits.txt")


def codes(s: str) -> np.ndarray:
    return np.searchsorted(np.frombuffer(b"ACGT", np.uint8),
                           np.frombuffer(s.encode(), np.uint8)).astype(np.uint8)


def cases():
    out = []
    for line in open(_PATH):
        line = line.strip()
        if not line.startswith("case"):
            continue
        _, genome, read, k, cap, total, hits = [x.strip() for x in line.split("|")]
        want = []
        for h in hits.split():
            p, s, d = h.split(":")
            want.append((int(p), 0 if s == "+" else 1, int(d)))
        out.append(dict(genome=genome, read=read, k=int(k), cap=int(cap),
                        total=int(total), hits=want))
    return out


def batch_of(read: str, k: int):
    words, off, lens = synth.pack_reads([codes(read)])
    return synth.ReadBatch(words, off, lens, np.array([k], np.uint8),
                           np.zeros(1, np.int64), np.zeros(1, np.uint8), np.zeros(1, np.int32))
