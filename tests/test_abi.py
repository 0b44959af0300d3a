"""The C-ABI library loads and exports every function include/mica.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import numpy as np
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
    assert p.hit_cap == 1000 and p.kernel == mica.KERNELS["bidirectional"]
    q = mica.IndexParams()
    lib.mica_index_params_default(ctypes.byref(q))
    assert (q.kmer_q, q.sa_sample, q.lower_bounds, q.full_sa) == (12, 16, 1, 1)
    bad = mica.IndexParams(12, 16, 1, 2)                      # full_sa is 0 or 1
    assert lib.mica_index_build_resident(b"ACGT", 4, ctypes.byref(bad), 0, ctypes.byref(ctypes.c_void_p())) == \
        mica.MICA_EINVAL


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
    # pipelined batches: arguments checked before any device call
    t = ctypes.c_uint64()
    assert lib.mica_align_submit(None, None, None, None, None, 0, None, ctypes.byref(t)) == mica.MICA_EINVAL
    assert lib.mica_align_collect(None, 1, ctypes.byref(ctypes.c_void_p())) == mica.MICA_EINVAL
    # the binding checks the host arrays' sizes before the library reads them
    idx = object.__new__(mica.Index)                  # no index: the check comes first
    words, off = np.zeros(4, np.uint32), np.array([0, 4], np.uint64)
    ln, kk = np.array([64], np.uint16), np.array([2], np.uint8)
    for args in ((words[:3], off, ln, kk), (words, off[:1], ln, kk), (words, off, ln, kk[:0])):
        for call in (idx.align, idx.submit):
            with pytest.raises(mica.MicaError) as e:
                call(*args)
            assert e.value.code == mica.MICA_EINVAL
    # defaults: pruning on, every placement reported
    p = mica.AlignParams()
    lib.mica_align_params_default(ctypes.byref(p))
    assert p.report == 0 and p.prune == 1


C_PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "mica.h"

/* argv: reference FASTA, reads FASTQ, output SAM.  Host-only calls: every
   read is written unmapped (an empty result). */
int main(int argc, char **argv)
{
    mica_reference *ref = NULL;
    mica_fastq *fq = NULL;
    mica_read_batch *b = NULL;
    mica_sam_writer *w = NULL;
    mica_read_batch_view v;
    mica_sam_params p;
    uint64_t *total, *offsets;
    if (argc != 4) return 9;
    if (mica_reference_read_fasta(argv[1], &ref) != MICA_OK) return 1;
    if (mica_fastq_open(argv[2], NULL, &fq) != MICA_OK) return 2;
    if (mica_fastq_read(fq, 1000, 2, &b) != MICA_OK) return 3;
    if (mica_read_batch_get_view(b, &v) != MICA_OK) return 4;
    total = calloc(v.n_reads, sizeof(uint64_t));
    offsets = calloc(v.n_reads + 1, sizeof(uint64_t));
    mica_sam_params_default(&p);
    if (mica_sam_open(argv[3], ref, &p, &w) != MICA_OK) return 5;
    if (mica_sam_write_batch(w, b, total, offsets, NULL, NULL) != MICA_OK) return 6;
    if (mica_sam_close(w) != MICA_OK) return 7;
    printf("%llu %s\n", (unsigned long long)v.n_reads, mica_strerror(MICA_EIO));
    free(total);
    free(offsets);
    mica_read_batch_free(b);
    mica_fastq_close(fq);
    mica_reference_free(ref);
    return 0;
}
"""


def test_c_program_uses_the_host_calls(lib, tmp_path):
    """A C99 program compiled against include/mica.h and linked with the
    library runs the host-only calls (FASTA, FASTQ, SAM) without a GPU."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "prog.c"
    src.write_text(C_PROGRAM)
    libdir = os.path.join(ROOT, "paper_1402_4876_gb300")
    exe = tmp_path / "prog"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"), str(src),
                    "-L" + libdir, "-lmica_gb300", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    (tmp_path / "ref.fa").write_bytes(b">chrA\nACGTACGTNNACGT\n>chrB\nTTTTGGGG\n")
    (tmp_path / "reads.fq").write_bytes(b"@q1 x\nACGTN\n+\nIIIII\n@q2\nGGGG\n+\n!!!!\n")
    out = subprocess.run([str(exe), str(tmp_path / "ref.fa"), str(tmp_path / "reads.fq"), str(tmp_path / "o.sam")],
                         capture_output=True, text=True, check=True)
    assert out.stdout.split()[0] == "2"
    lines = (tmp_path / "o.sam").read_text().splitlines()
    assert lines[:3] == ["@HD\tVN:1.6\tSO:unsorted", "@SQ\tSN:chrA\tLN:14", "@SQ\tSN:chrB\tLN:8"]
    assert lines[-2:] == ["q1\t4\t*\t0\t0\t*\t*\t0\t0\tACGTN\tIIIII", "q2\t4\t*\t0\t0\t*\t*\t0\t0\tGGGG\t!!!!"]


class _IndexHeader(ctypes.Structure):
    """The index file's leading header as the library writes it (version 5):
    magic, version, q, sampling, flags (version 5: bit 0 = the whole suffix
    array is kept), the text's sizes and the short-suffix codes."""
    _fields_ = [("magic", ctypes.c_char * 8), ("version", ctypes.c_uint32), ("kmer_q", ctypes.c_uint32),
                ("sa_sample", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("dollar_row", ctypes.c_uint64), ("C", ctypes.c_uint64 * 5), ("n_occ_blocks", ctypes.c_uint64),
                ("n_super", ctypes.c_uint64), ("n_mark_blocks", ctypes.c_uint64), ("n_samples", ctypes.c_uint64),
                ("table_len", ctypes.c_uint64), ("nshort", ctypes.c_uint32), ("short_pad", ctypes.c_uint32 * 12),
                ("short_len", ctypes.c_uint32 * 12)]


def _consistent_header(n=1000, q=8, s=16):
    h = _IndexHeader()
    h.magic, h.version, h.kmer_q, h.sa_sample, h.n = b"MICAIDX1", 3, q, s, n   # a version-3 file: no table block
    h.n_occ_blocks = (n + 1) // 96 + 1
    h.n_super = (h.n_occ_blocks + 681) // 682
    h.n_mark_blocks = (n + 1) // 480 + 1
    h.n_samples = (n + 1) // s + 1
    h.table_len = (1 << (2 * q)) + 1
    h.nshort = min(q, n + 1)
    return h


@pytest.mark.parametrize("field,value", [
    ("magic", b"MICAIDX9"), ("version", 6), ("kmer_q", 0), ("kmer_q", 13), ("sa_sample", 0), ("flags", 1),
    ("n_occ_blocks", 5), ("n_super", 0), ("n_mark_blocks", 0), ("table_len", 17), ("n_samples", 2000),
    ("nshort", 3), ("n", 1 << 32),
])
def test_index_file_header_checked_before_any_device_call(tmp_path, field, value):
    """A malformed index header is MICA_EIO before the library touches a GPU."""
    import paper_1402_4876_gb300 as mica
    lib = mica.lib()
    h = _consistent_header()
    setattr(h, field, value)
    path = tmp_path / "bad.mica"
    path.write_bytes(bytes(h) + bytes(64))
    out = ctypes.c_void_p()
    assert lib.mica_index_load(str(path).encode(), 0, ctypes.byref(out)) == mica.MICA_EIO
    # the unmodified header passes the checks: without a device the load then
    # stops at the device call itself
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        path.write_bytes(bytes(_consistent_header()) + bytes(64))
        assert lib.mica_index_load(str(path).encode(), 0, ctypes.byref(out)) == mica.MICA_ECUDA
    for blob in (b"", b"MICAIDX1", bytes(h)[:40]):          # empty and truncated files
        path.write_bytes(blob)
        assert lib.mica_index_load(str(path).encode(), 0, ctypes.byref(out)) == mica.MICA_EIO


def test_index_file_flags_checked(tmp_path):
    """Version 5 headers carry flags (bit 0 alone is defined); earlier versions
    must have the field zero."""
    import paper_1402_4876_gb300 as mica
    lib = mica.lib()
    out = ctypes.c_void_p()
    path = tmp_path / "bad.mica"
    for version, flags in ((5, 2), (5, 0x80000001), (4, 1), (2, 1)):
        h = _consistent_header()
        h.version, h.flags = version, flags
        path.write_bytes(bytes(h) + bytes(4096))
        assert lib.mica_index_load(str(path).encode(), 0, ctypes.byref(out)) == mica.MICA_EIO, (version, flags)


def test_shape_table_and_defaults_need_no_gpu():
    import paper_1402_4876_gb300 as mica
    lib = mica.lib()
    shapes = mica.tuning_shapes()
    assert len(shapes) == lib.mica_tuning_shapes() >= 1
    assert shapes[0] == (256, 8, 3)           # the default persistent shape
    for stack, warps, min_ctas in shapes:
        assert stack in (128, 256) and warps in (4, 8) and 1 <= min_ctas <= 8
    a = ctypes.c_int()
    assert lib.mica_tuning_shape_info(len(shapes), ctypes.byref(a), ctypes.byref(a), ctypes.byref(a)) \
        == mica.MICA_EINVAL
    sp = mica.ServerParams()
    lib.mica_server_params_default(ctypes.byref(sp))
    assert (sp.max_device_bytes, sp.max_tick_reads, sp.hit_cap, sp.kernel, sp.workers, sp.start_paused,
            sp.chunk_reads) == (0, 1 << 20, 1000, mica.KERNELS["bidirectional"], 2, 0, 1 << 18)
    wp = mica.SamParams(b"x", 1, b"y", 7)
    lib.mica_sam_params_default(ctypes.byref(wp))
    assert (wp.qname_prefix, wp.secondary, wp.command_line, wp.threads) == (None, 0, None, 0)
