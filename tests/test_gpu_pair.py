"""Mate pairing on the GPU (mica_pair_batch / mica_pair_device) equals the
oracle's pairing of the same hit lists: on hand-built lists with ties and
window edges, on the oracle's result for paired reads of the 64 Mbp repeat
genome, and on the GPU's own result (device path, torch tensors)."""
import numpy as np
import pytest

import oracle
import synth
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu


def _rows(arr):
    return [(int(x["n_concordant"]), int(x["n_best"]), int(x["pos_plus"]), int(x["pos_minus"]),
             int(x["plus_mate"]), int(x["mm"])) for x in arr]


class _Hits:
    def __init__(self, lists):
        self.lists = [sorted(x, key=lambda h: (h[0], h[1])) for x in lists]
        self.offsets = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.uint64)
        m = gc.mica()
        flat = [h for x in self.lists for h in x]
        self.hits = np.zeros(len(flat), dtype=m.HIT_DTYPE)
        for j, (p, s, d) in enumerate(flat):
            self.hits[j] = (p, s, d, 0)

    def as_tuples(self, i):
        return self.lists[i]


def test_random_hit_lists_equal_oracle():
    rng = np.random.default_rng(5)
    lists, lens = [], []
    for p in range(400):
        for mate in range(2):
            n = int(rng.integers(0, 12))
            pos = rng.integers(0, 5_000, size=n)
            lists.append({(int(x), int(rng.integers(0, 2)), int(rng.integers(0, 3))) for x in pos})
            lens.append(int(rng.choice([100, 150, 250])))
    lists = [sorted(x) for x in lists]
    r = _Hits(lists)
    lens = np.array(lens, np.uint16)
    for lo, hi in ((300, 700), (0, 5_000), (450, 450)):
        got = gc.mica().pair_batch(r, lens, lo, hi)
        assert _rows(got) == oracle.pair(r, lens, lo, hi), (lo, hi)


def test_paired_reads_64m_equal_oracle_and_device_path():
    import torch
    m = gc.mica()
    g = gc.genome("64m")
    b = synth.paired_reads(g.codes, 3_000, seed=91)
    want_hits = gc.oracle_index("64m").align(b, cap=1000)
    want = oracle.pair(want_hits, b.lengths, 300, 700)
    idx = gc.gpu_index("64m")
    res = idx.align_batch(b, hit_cap=1000)
    gc.assert_same(res, want_hits)
    assert _rows(m.pair_batch(res, b.lengths, 300, 700)) == want
    # a pair is found when both mates carry <= 2 of their ~1% substitutions:
    # P = (sum_{j<=2} Binom(150, 0.01)(j))^2 = 0.809^2 = 0.655 (repeats add a little)
    assert 0.60 < np.mean([w[0] > 0 for w in want]) < 0.72
    # device path on the device result of the same batch
    dev = torch.device("cuda", 0)
    d = (torch.from_numpy(b.words.view(np.int32)).to(dev), torch.from_numpy(b.word_off.view(np.int64)).to(dev),
         torch.from_numpy(b.lengths.view(np.int16)).to(dev), torch.from_numpy(b.k).to(dev))
    r = idx.align_device(*d, b.n, hit_cap=1000)
    t, o, h = r.tensors()
    out = torch.zeros(b.n // 2 * 20, dtype=torch.uint8, device=dev)
    m.pair_device(o, h, d[2], b.n // 2, 300, 700, out)
    torch.cuda.synchronize()
    assert _rows(out.cpu().numpy().view(m.PAIR_DTYPE)) == want
