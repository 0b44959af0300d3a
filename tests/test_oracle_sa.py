"""Pins for the oracle's suffix arrays (sorting and SA-IS)."""
import numpy as np
import pytest

import oracle
import synth
from tests import refcheck


def _fib_word(n):
    a, b = [0], [0, 1]          # Fibonacci word over {A, C}
    while len(b) < n:
        a, b = b, b + a
    return np.array(b[:n], dtype=np.uint8)


def _strings():
    rng = np.random.default_rng(7)
    out = [np.zeros(0, np.uint8), np.array([2], np.uint8), np.array([0, 0], np.uint8)]
    for n in (3, 5, 17, 64, 200):
        out.append(rng.integers(0, 4, n).astype(np.uint8))
        out.append(rng.integers(0, 2, n).astype(np.uint8))     # two-letter
    for n in (1, 2, 31, 100):
        out.append(np.zeros(n, np.uint8))                      # all-A
        out.append(np.full(n, 3, np.uint8))                    # all-T
        out.append(np.resize(np.array([0, 1], np.uint8), n))   # (AC)^n
        out.append(np.resize(np.array([3, 0, 2], np.uint8), n))
    out.append(_fib_word(150))
    return out


@pytest.mark.parametrize("idx", range(len(_strings())))
def test_sa_matches_definition(idx):
    g = _strings()[idx]
    want = refcheck.suffix_array_by_definition(g)
    assert np.array_equal(oracle.sa_sort(g), want)
    assert np.array_equal(oracle.sa_is(g), want)


def test_handworked_sa_and_bwt():
    # tests/golden/handworked_sa.txt: G = ACGTTGCA worked out by hand
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "handworked_sa.txt")
    vals = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split("=", 1)
            vals[k.strip()] = v.strip()
    g = np.frombuffer(vals["genome"].encode(), np.uint8)
    codes = np.searchsorted(np.frombuffer(b"ACGT", np.uint8), g).astype(np.uint8)
    sa = [int(x) for x in vals["sa"].split()]
    assert oracle.sa_sort(codes).tolist() == sa
    assert oracle.sa_is(codes).tolist() == sa
    fm = oracle.FMIndex(codes)
    bwt = "".join("ACGT$"[c] for c in fm.bwt())
    assert bwt == vals["bwt"]
    assert [fm.C(c) for c in range(4)] == [int(x) for x in vals["C"].split()]


@pytest.mark.parametrize("kind", ["random", "periodic", "repeats"])
def test_sais_equals_sort_larger(kind):
    rng = np.random.default_rng(3)
    if kind == "random":
        g = rng.integers(0, 4, 100_000).astype(np.uint8)
    elif kind == "periodic":
        g = np.resize(rng.integers(0, 4, 7).astype(np.uint8), 20_000)
    else:
        g = synth.repeat_genome(60_000, 5, copy_frac=0.2, copy_len=(500, 3000),
                                tandem_frac=0.1, array_len=(100, 2000)).codes
    a = oracle.sa_sort(g)
    b = oracle.sa_is(g)
    assert np.array_equal(a, b)
    # a permutation of 0..N
    assert np.array_equal(np.sort(a), np.arange(len(g) + 1, dtype=np.uint32))
