"""Serving loop: continuous batching over a resident index.  Each request's
result is bit-identical alone (mica_align_batch) and in the mix, and equal to
the oracle; admission, cancellation and budget refusal are exercised on the
host side of the server."""
import threading
import time

import numpy as np
import pytest

import synth
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu


def _requests(n_req, seed):
    g = gc.genome("64m")
    full = synth.reads_uneven(g, n=200_000)
    rng = np.random.default_rng(seed)
    out, start = [], 0
    for _ in range(n_req):
        size = int(rng.choice([1, 7, 100, 1000, 5000, 20000]))
        idx = np.arange(start, start + size) % full.n
        start += size
        out.append(full.subset(idx))
    return out


def test_alone_equals_mix_equals_oracle():
    idx = gc.gpu_index("64m")
    reqs = _requests(24, 1)
    alone = [idx.align_batch(r, hit_cap=1000) for r in reqs]
    results = [None] * len(reqs)
    # chunks of 3,000 reads: the larger requests run over several ticks
    with gc.mica().Server(idx, hit_cap=1000, workers=2, max_tick_reads=30000, chunk_reads=3000) as srv:
        ids = [None] * len(reqs)
        rng = np.random.default_rng(2)

        def client(j0):
            for j in range(j0, len(reqs), 3):
                time.sleep(float(rng.exponential(0.002)))
                ids[j] = srv.submit_batch(reqs[j])

        th = [threading.Thread(target=client, args=(j,)) for j in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for j, rid in enumerate(ids):
            results[j], lat = srv.wait(rid)
            assert lat >= 0
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        n_chunks = sum(max(1, -(-r.n // 3000)) for r in reqs)
        assert st["ticks"] < n_chunks             # chunks of several requests shared launches
    for j, r in enumerate(reqs):
        gc.assert_same(results[j], alone[j], f"request {j}")
    fm = gc.oracle_index("64m")
    for j in (0, 5, 11):
        gc.assert_same(results[j], fm.align(reqs[j], cap=1000), f"oracle {j}")


def test_paused_admission_cancel_and_timeout():
    idx = gc.gpu_index("64m")
    reqs = _requests(4, 3)
    m = gc.mica()
    with m.Server(idx, workers=1, start_paused=True) as srv:
        ids = [srv.submit_batch(r) for r in reqs]
        assert srv.stats()["pending"] == 4
        assert srv.poll(ids[0]) is None
        with pytest.raises(m.MicaError) as e:
            srv.wait(ids[0], timeout_ms=50)
        assert e.value.code == m.MICA_ETIMEOUT
        assert srv.cancel(ids[1]) == 0
        assert srv.cancel(ids[1]) == m.MICA_ENOTFOUND
        srv.resume()
        for j in (0, 2, 3):
            res, _ = srv.wait(ids[j])
            gc.assert_same(res, idx.align_batch(reqs[j], hit_cap=1000))
        st = srv.stats()
        assert st["cancelled"] == 1 and st["completed"] == 3


def test_budget_refusal_and_serialised_admission():
    """Admission charges each tick the workspace its reads need
    (mica_server_workspace_bytes) against the worker's share of the budget:
    with a share that holds a tick of 5,000 reads, larger requests run in
    smaller chunks and still equal their alone results, and the workspace in
    use never exceeds the budget; a share that cannot hold a one-read tick
    refuses every request."""
    idx = gc.gpu_index("64m")
    m = gc.mica()
    reqs = _requests(6, 4)
    assert max(r.n for r in reqs) > 5000
    share = m.Server.workspace_bytes(idx, 5000, 5000 * 16)
    assert share > m.Server.workspace_bytes(idx, 1000, 1000 * 16) > m.Server.workspace_bytes(idx, 1, 16)
    with m.Server(idx, workers=2, max_device_bytes=2 * share) as srv:
        ids = [srv.submit_batch(r) for r in reqs]
        for r, rid in zip(reqs, ids):
            res, _ = srv.wait(rid)
            gc.assert_same(res, idx.align_batch(r, hit_cap=1000))
            assert 0 < srv.stats()["device_bytes_in_use"] <= 2 * share
        assert srv.stats()["ticks"] >= sum(-(-r.n // 5000) for r in reqs) // 2
    tiny = m.Server.workspace_bytes(idx, 1, 16) // 2
    with m.Server(idx, workers=1, max_device_bytes=tiny) as srv:
        with pytest.raises(m.MicaError) as e:
            srv.submit_batch(reqs[0])
        assert e.value.code == m.MICA_ENOMEM


def test_invalid_request_and_stop_with_queue():
    idx = gc.gpu_index("64m")
    m = gc.mica()
    srv = m.Server(idx, workers=1, start_paused=True)
    with pytest.raises(m.MicaError) as e:
        srv.submit(np.zeros(4, np.uint32), np.array([0, 4], np.uint64), np.array([10], np.uint16),
                   np.array([4], np.uint8))
    assert e.value.code == m.MICA_EINVAL
    for r in _requests(3, 5):
        srv.submit_batch(r)
    srv.stop()          # drops the queued requests, joins the workers
    # a request with chunks already on the GPU is finished, not dropped, by stop
    big = _requests(6, 4)
    srv = m.Server(idx, workers=1, chunk_reads=1000)
    rid = srv.submit_batch(max(big, key=lambda r: r.n))
    srv.stop()
