"""Bounded device waits (the paper's give-up rule of Section 2 kept as a
bound on every wait): with a tiny idle bound, warps that find no work while
others are still searching give up, the launch stops, and the call returns
MICA_ETIMEOUT with no trap; the index stays usable and the next call, with
the default bounds, equals the oracle."""
import numpy as np
import pytest

import synth
from tests import gpu_common as gc

pytestmark = pytest.mark.gpu


def test_idle_bound_times_out_and_the_index_stays_usable():
    m = gc.mica()
    g = gc.genome("64m")
    # 20,000 reads of uneven length and budget: 40,000 tasks leave most of the
    # persistent grid's warps without work while the rest still search
    b = synth.reads_uneven(g, n=200_000).subset(np.arange(0, 200_000, 10))
    idx = gc.gpu_index("64m")
    want = gc.oracle_index("64m").align(b, cap=1000)
    try:
        idx.set_wait_limits(idle_rounds=1)
        for report in ("all", "best_stratum"):          # the captured-graph path and the deepening path
            with pytest.raises(m.MicaError) as e:
                idx.align_batch(b, hit_cap=1000, kernel="persistent", report=report)
            assert e.value.code == m.MICA_ETIMEOUT, report
    finally:
        idx.set_wait_limits()
    for call in range(2):
        gc.assert_same(idx.align_batch(b, hit_cap=1000, kernel="persistent"), want, f"after timeout, call {call}")
