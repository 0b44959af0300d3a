"""Shared fixtures for the GPU parity tests (CUDA path vs the CPU oracle)."""
import functools

import numpy as np

import oracle
import synth


def mica():
    import paper_1402_4876_gb300 as m
    return m


@functools.lru_cache(maxsize=None)
def genome(name):
    if name == "1m":
        return synth.genome_1m()
    if name == "64m":
        return synth.genome_64m()
    raise KeyError(name)


@functools.lru_cache(maxsize=None)
def oracle_index(name):
    g = genome(name).codes
    return oracle.FMIndex(g, "sort" if g.size <= 200_000 else "sais")


@functools.lru_cache(maxsize=None)
def gpu_index(name, kmer_q=12, sa_sample=16):
    return mica().Index.build(synth.to_acgt_bytes(genome(name).codes), kmer_q=kmer_q, sa_sample=sa_sample)


def assert_same(got, want, ctx=""):
    """Bit-exact: totals, CSR offsets and every (pos, strand, mm) in order."""
    assert np.array_equal(got.total, want.total), f"{ctx}: totals differ at {np.flatnonzero(got.total != want.total)[:10]}"
    assert np.array_equal(got.offsets, want.offsets), f"{ctx}: offsets differ"
    g = got.hits[["pos", "strand", "mm"]]
    w = want.hits[["pos", "strand", "mm"]]
    bad = np.flatnonzero(g != w)
    assert bad.size == 0, f"{ctx}: {bad.size} hits differ, first at {bad[:5]}"


def batch_from_reads(reads, ks):
    words, off, lens = synth.pack_reads(reads)
    n = len(reads)
    return synth.ReadBatch(words, off, lens, np.asarray(ks, np.uint8), np.zeros(n, np.int64),
                           np.zeros(n, np.uint8), np.zeros(n, np.int32))
