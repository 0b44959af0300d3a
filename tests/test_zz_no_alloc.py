"""mica_offsets_noalloc: the hit-list offsets for callers that may not
allocate device memory (graph capture, foreign allocators, fixed-footprint
services) must equal the offsets the regular device entry point returns.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh
process."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


class _View:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def test_offsets_without_allocation_equal_align_device():
    import torch

    import paper_1402_4876_gb300 as mica

    g = synth.repeat_genome(2_000_000, 7, copy_frac=0.2, copy_len=(500, 5000), tandem_frac=0.05,
                            array_len=(100, 2000))
    reads = synth.sample_reads(g, np.full(20_000, 100), np.full(20_000, 2), np.random.default_rng(5),
                               subs="rate", sub_rate=0.01, repeat_frac=0.3)
    idx = mica.Index.build(synth.to_acgt_bytes(g.codes), kmer_q=12, sa_sample=16)
    dev = torch.device("cuda", 0)
    dw = torch.from_numpy(reads.words.view(np.int32)).to(dev)
    do = torch.from_numpy(reads.word_off.view(np.int64)).to(dev)
    dl = torch.from_numpy(reads.lengths.view(np.int16)).to(dev)
    dk = torch.from_numpy(reads.k).to(dev)
    res = idx.align_device(dw, do, dl, dk, reads.n, hit_cap=1000)
    n = res.n_reads
    want = torch.as_tensor(_View(res._r.offsets, n + 1, "<i8"), device=dev).clone()
    counts = want[1:] - want[:-1]
    assert int(counts.max()) > 1 and int(want[-1]) == res.n_hits        # a varied workload
    for call in range(2):                                              # the scratch keeps old contents
        out = torch.full((n + 1,), -1, dtype=torch.int64, device=dev)
        mica.offsets_noalloc(counts, n, out)
        torch.cuda.synchronize()
        assert torch.equal(out, want), f"call {call}"
    # beyond the scratch array's room: rejected before any work
    with pytest.raises(mica.MicaError) as e:
        mica.offsets_noalloc(counts, mica.NOALLOC_MAX_COUNTS + 1, out)
    assert e.value.code == mica.MICA_EINVAL
    # a counts tensor of the wrong element size or length is refused by the binding
    with pytest.raises(mica.MicaError) as e:
        mica.offsets_noalloc(counts.to(torch.int32), n, out)
    assert e.value.code == mica.MICA_EINVAL
    with pytest.raises(mica.MicaError) as e:
        mica.offsets_noalloc(counts[:-1], n, out)
    assert e.value.code == mica.MICA_EINVAL
    idx.free()


@pytest.mark.parametrize("n", [0, 1, 2047, 2048, 2049, 3 * 2048 + 5])
def test_offsets_without_allocation_at_tile_edges(n):
    """Empty input, one count, and counts at and around the 2,048-count tile
    size, against numpy's running sum."""
    import torch

    import paper_1402_4876_gb300 as mica

    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(100 + n)
    c = rng.integers(0, 1 << 20, size=n, dtype=np.int64)
    want = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(c, out=want[1:])
    counts = torch.from_numpy(c).to(dev)
    for call in range(2):
        out = torch.full((n + 1,), -1, dtype=torch.int64, device=dev)
        mica.offsets_noalloc(counts, n, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want), f"n={n} call {call}"
