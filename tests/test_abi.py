"""The C-ABI library loads and exports every function include/mica.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mica.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mica_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location("mica_build", os.path.join(ROOT, "paper_1402_4876_gb300", "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = mod.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    import paper_1402_4876_gb300 as mica
    assert set(_declared()) <= set(mica.exported_symbols())


def test_strerror_and_defaults(lib):
    import paper_1402_4876_gb300 as mica
    lib = mica.lib()
    assert lib.mica_strerror(0) == b"ok"
    assert b"invalid" in lib.mica_strerror(-1)
    p = mica.AlignParams()
    lib.mica_align_params_default(ctypes.byref(p))
    assert p.hit_cap == 1000 and p.kernel == 0
    q = mica.IndexParams()
    lib.mica_index_params_default(ctypes.byref(q))
    assert (q.kmer_q, q.sa_sample) == (12, 16)


def test_host_side_rejections_need_no_gpu():
    import paper_1402_4876_gb300 as mica
    lib = mica.lib()
    out = ctypes.c_void_p()
    # bad index parameters and a non-ACGT genome are rejected before any CUDA call
    bad = mica.IndexParams(13, 16)
    g = b"ACGTN"
    assert lib.mica_index_build_resident(g, 4, ctypes.byref(bad), 0, ctypes.byref(out)) == mica.MICA_EINVAL
    ok = mica.IndexParams(8, 16)
    assert lib.mica_index_build_resident(g, 5, ctypes.byref(ok), 0, ctypes.byref(out)) == mica.MICA_EINVAL
    assert lib.mica_index_load(b"/nonexistent/index", 0, ctypes.byref(out)) == mica.MICA_EIO
    # the gather ceiling checks its sizes before touching a device
    gbs = ctypes.c_double()
    assert lib.mica_gather_ceiling(0, 1 << 20, 24, 1 << 20, 1, ctypes.byref(gbs), None) == mica.MICA_EINVAL
    assert lib.mica_gather_ceiling(0, 1000, 32, 1 << 20, 1, ctypes.byref(gbs), None) == mica.MICA_EINVAL
    assert lib.mica_gather_ceiling(0, 1 << 20, 32, 1 << 20, 1, None, None) == mica.MICA_EINVAL
    # pairing rejects an inverted insert window before touching a device
    assert lib.mica_pair_batch(0, None, None, None, 1, 700, 300, None) == mica.MICA_EINVAL
    assert lib.mica_pair_device(None, None, None, 1, 700, 300, None, None) == mica.MICA_EINVAL
    # defaults: pruning on, every placement reported
    p = mica.AlignParams()
    lib.mica_align_params_default(ctypes.byref(p))
    assert p.report == 0 and p.prune == 1
