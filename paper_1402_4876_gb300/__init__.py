"""GB300 k-mismatch FM-index read search (the BWT phase of MICA, Section 2).

Thin ctypes binding over ``libmica_gb300.so`` (C ABI in ``include/mica.h``).
Every step of the search runs in the library's CUDA kernels; this module only
marshals arguments.  There is no CPU fallback: if the library is missing or
cannot be loaded, importing the binding raises.

    import paper_1402_4876_gb300 as mica
    idx = mica.Index.build(genome_acgt_bytes)            # resident on cuda:0
    res = idx.align(words, word_off, lengths, k, hit_cap=1000)
    res.hits_of(i)  # [(pos, strand, mismatches), ...]
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmica_gb300.so")

MICA_OK = 0
MICA_EINVAL = -1
MICA_ENOMEM = -2
MICA_EIO = -3
MICA_ECUDA = -4
MICA_ETIMEOUT = -5
MICA_EINTERNAL = -6
MICA_EBUSY = -7
MICA_ENOTFOUND = -8
MAX_READ_LEN = 256
KERNELS = {"persistent": 0, "plain": 1, "plain_by_length": 2, "bidirectional": 3}
REPORTS = {"all": 0, "best_stratum": 1}

HIT_DTYPE = np.dtype([("pos", "<u4"), ("strand", "u1"), ("mm", "u1"), ("pad", "<u2")])


class MicaError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_lib.mica_strerror(code).decode()} ({code})")


class IndexParams(ctypes.Structure):
    _fields_ = [("kmer_q", ctypes.c_uint32), ("sa_sample", ctypes.c_uint32), ("lower_bounds", ctypes.c_uint32),
                ("full_sa", ctypes.c_uint32)]


class AlignParams(ctypes.Structure):
    _fields_ = [("hit_cap", ctypes.c_uint32), ("kernel", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
                ("prune", ctypes.c_uint32), ("report", ctypes.c_uint32)]


class _Result(ctypes.Structure):
    _fields_ = [("n_reads", ctypes.c_uint64), ("total", ctypes.POINTER(ctypes.c_uint64)),
                ("offsets", ctypes.POINTER(ctypes.c_uint64)), ("hits", ctypes.c_void_p)]


class _DeviceResult(ctypes.Structure):
    _fields_ = [("n_reads", ctypes.c_uint64), ("n_hits", ctypes.c_uint64), ("total", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p), ("hits", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in
                ("tasks", "seeds", "nodes", "rank_blocks", "intervals", "located", "lf_steps",
                 "spills", "retries", "launches", "warp_rounds", "lane_ops", "rounds_multi", "rounds_single",
                 "rounds_seed", "graph_captures", "graph_replays", "graph_fallbacks", "lb_steps",
                 "lb_dead_tasks", "queue_wait_ns", "idle_wait_ns", "overflow_moves", "grid_ctas", "fallback_reads",
                 "verified", "verify_bytes", "verify_sectors")] + [("search_ms", ctypes.c_float), ("kernel_ms", ctypes.c_float),
                                                      ("total_ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("plain_block", ctypes.c_uint32), ("plain_budget", ctypes.c_uint32),
                ("plain_block_len", ctypes.c_uint32 * 4), ("prefetch", ctypes.c_int32),
                ("bidir_budget", ctypes.c_uint32), ("bidir_verify", ctypes.c_uint32), ("bidir_shape", ctypes.c_int32)]


def tuning_shapes() -> list:
    """[(stack_nodes, warps_per_cta, min_ctas_per_sm)] of the compiled persistent kernel shapes."""
    out = []
    for i in range(_lib.mica_tuning_shapes()):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.mica_tuning_shape_info(i, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "mica_tuning_shape_info")
        out.append((a.value, b.value, c.value))
    return out


class ServerParams(ctypes.Structure):
    _fields_ = [("max_device_bytes", ctypes.c_uint64), ("max_tick_reads", ctypes.c_uint64),
                ("hit_cap", ctypes.c_uint32), ("kernel", ctypes.c_int32), ("workers", ctypes.c_int32),
                ("start_paused", ctypes.c_int32), ("chunk_reads", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in
                ("submitted", "completed", "failed", "cancelled", "ticks", "reads", "pending",
                 "device_bytes_in_use", "device_budget")] + [("busy_s", ctypes.c_double)]


class IndexInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("rows", ctypes.c_uint64), ("kmer_q", ctypes.c_uint32),
                ("sa_sample", ctypes.c_uint32), ("dollar_row", ctypes.c_uint64),
                ("C", ctypes.c_uint64 * 5), ("occ_bytes", ctypes.c_uint64), ("mark_bytes", ctypes.c_uint64),
                ("sample_bytes", ctypes.c_uint64), ("table_bytes", ctypes.c_uint64), ("device", ctypes.c_int32),
                ("lower_bounds", ctypes.c_uint32), ("rev_occ_bytes", ctypes.c_uint64),
                ("rev_table_bytes", ctypes.c_uint64), ("full_sa", ctypes.c_uint32),
                ("full_sa_bytes", ctypes.c_uint64), ("long_q", ctypes.c_uint32),
                ("long_table_bytes", ctypes.c_uint64)]


# exported symbol -> (restype, argtypes); the C ABI's full surface
P = ctypes.c_void_p
_u64, _u32, _i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
SIGNATURES = {
    "mica_strerror": (ctypes.c_char_p, [_i32]),
    "mica_index_params_default": (None, [P]),
    "mica_align_params_default": (None, [P]),
    "mica_index_build_resident": (_i32, [P, _u64, P, _i32, P]),
    "mica_index_build": (_i32, [P, _u64, P, ctypes.c_char_p]),
    "mica_index_save": (_i32, [P, ctypes.c_char_p]),
    "mica_index_load": (_i32, [ctypes.c_char_p, _i32, P]),
    "mica_index_free": (None, [P]),
    "mica_index_get_info": (_i32, [P, P]),
    "mica_align_batch": (_i32, [P, P, P, P, P, _u64, P, P]),
    "mica_result_free": (None, [P]),
    "mica_align_submit": (_i32, [P, P, P, P, P, _u64, P, P]),
    "mica_align_collect": (_i32, [P, _u64, P]),
    "mica_align_device": (_i32, [P, P, P, P, P, _u64, P, P]),
    "mica_get_stats": (_i32, [P, P]),
    "mica_debug_suffix_array": (_i32, [P, _u64, _i32, P]),
    "mica_debug_occ": (_i32, [P, P, _u64, P]),
    "mica_debug_locate": (_i32, [P, P, _u64, P]),
    "mica_debug_full_sa": (_i32, [P, ctypes.c_uint32, _u64, _u64, P]),
    "mica_debug_table_interval": (_i32, [P, ctypes.c_uint32, P, ctypes.c_uint32, _u64, P]),
    "mica_debug_seed_interval": (_i32, [P, P, _u32, _u64, P]),
    "mica_tuning_shapes": (_i32, []),
    "mica_tuning_shape_info": (_i32, [_i32, P, P, P]),
    "mica_set_tuning": (_i32, [P, P]),
    "mica_get_tuning": (_i32, [P, P]),
    "mica_set_wait_limits": (_i32, [P, _u32, _u32]),
    "mica_autotune": (_i32, [P, P, P, P, P, _u64, _u32, _u32, P]),
    "mica_tuning_cache_store": (_i32, [ctypes.c_char_p, P, _u32, _u32, P]),
    "mica_tuning_cache_lookup": (_i32, [ctypes.c_char_p, P, _u32, _u32, P]),
    "mica_offsets_noalloc": (_i32, [P, _u64, P, P]),
    "mica_gather_ceiling": (_i32, [ctypes.c_int, _u64, _u32, _u64, _u32, P, P]),
    "mica_debug_lower_bounds": (_i32, [P, P, P, P, P, _u64, P]),
    "mica_pair_device": (_i32, [P, P, P, _u64, _u32, _u32, P, P]),
    "mica_pair_batch": (_i32, [ctypes.c_int, P, P, P, _u64, _u32, _u32, P]),
    "mica_reference_create": (_i32, [P, _u64, P, P, _u64, P]),
    "mica_reference_read_fasta": (_i32, [ctypes.c_char_p, P]),
    "mica_reference_save": (_i32, [P, ctypes.c_char_p]),
    "mica_reference_load": (_i32, [ctypes.c_char_p, P]),
    "mica_reference_free": (None, [P]),
    "mica_reference_get_info": (_i32, [P, P]),
    "mica_reference_text": (_i32, [P, P, P]),
    "mica_reference_contig": (_i32, [P, _u64, P, P, P]),
    "mica_reference_ambiguous_run": (_i32, [P, _u64, P, P]),
    "mica_reference_locate": (_i32, [P, P, P, _u64, P, P]),
    "mica_reference_filter": (_i32, [P, P, _u64, P, P, P, P]),
    "mica_fastq_open": (_i32, [ctypes.c_char_p, ctypes.c_char_p, P]),
    "mica_fastq_read": (_i32, [P, _u64, ctypes.c_uint8, P]),
    "mica_fastq_close": (None, [P]),
    "mica_read_batch_get_view": (_i32, [P, P]),
    "mica_read_batch_read": (_i32, [P, _u64, P, P, P, P]),
    "mica_read_batch_free": (None, [P]),
    "mica_read_batch_filter_n": (_i32, [P, P, P, P, P, P]),
    "mica_sam_write_batch": (_i32, [P, P, P, P, P, P]),
    "mica_sam_params_default": (None, [P]),
    "mica_sam_open": (_i32, [ctypes.c_char_p, P, P, P]),
    "mica_sam_write": (_i32, [P, P, P, P, _u64, P, P, P, P]),
    "mica_sam_close": (_i32, [P]),
    "mica_server_params_default": (None, [P]),
    "mica_server_start": (_i32, [P, P, P]),
    "mica_server_workspace_bytes": (_i32, [P, _u64, _u64, P]),
    "mica_server_submit": (_i32, [P, P, P, P, P, _u64, P]),
    "mica_server_poll": (_i32, [P, _u64, P, P]),
    "mica_server_wait": (_i32, [P, _u64, _u32, P, P]),
    "mica_server_cancel": (_i32, [P, _u64]),
    "mica_server_resume": (None, [P]),
    "mica_server_get_stats": (_i32, [P, P]),
    "mica_server_stop": (None, [P]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_1402_4876_gb300/_build.py` "
                          "or __graft_entry__.build() (nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


def _check(rc: int, what: str):
    if rc != MICA_OK:
        raise MicaError(rc, what)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _acgt(genome) -> np.ndarray:
    if isinstance(genome, (bytes, bytearray)):
        return np.frombuffer(bytes(genome), dtype=np.uint8)
    return np.ascontiguousarray(genome, dtype=np.uint8)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)   # torch.cuda.Stream


class Result:
    """Host-side hit lists in CSR form."""

    def __init__(self, total, offsets, hits):
        self.total = total
        self.offsets = offsets
        self.hits = hits

    def read_hits(self, i: int) -> np.ndarray:
        return self.hits[int(self.offsets[i]):int(self.offsets[i + 1])]

    def hits_of(self, i: int) -> list:
        h = self.read_hits(i)
        return [(int(p), int(s), int(d)) for p, s, d in zip(h["pos"], h["strand"], h["mm"])]


class _ResultOwner:
    """Frees a library-owned mica_result once no numpy view of it is left."""

    def __init__(self, out):
        self._out = out

    def __del__(self):
        if self._out is not None and _lib is not None:
            _lib.mica_result_free(self._out)
            self._out = None


def _view(addr: int, n: int, dtype, owner) -> np.ndarray:
    dtype = np.dtype(dtype)
    if n == 0 or not addr:
        return np.empty(0, dtype=dtype)
    buf = (ctypes.c_char * (n * dtype.itemsize)).from_address(addr)
    buf._owner = owner                       # the views keep the result alive
    return np.frombuffer(buf, dtype=dtype)


def _take_result(out) -> Result:
    """Numpy views (no copy) of a library-owned mica_result; the result is
    freed when the last view is collected."""
    owner = _ResultOwner(out)
    r = out.contents
    n = int(r.n_reads)
    offsets = _view(ctypes.cast(r.offsets, ctypes.c_void_p).value, n + 1, np.uint64, owner)
    total = _view(ctypes.cast(r.total, ctypes.c_void_p).value, n, np.uint64, owner)
    nh = int(offsets[-1]) if n else 0
    hits = _view(r.hits, nh, HIT_DTYPE, owner)
    if hits.size == 0:
        hits = np.empty(0, dtype=HIT_DTYPE)
    return Result(total, offsets, hits)


class _CudaArray:
    """Zero-copy view of a device array for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3, "strides": None}


class DeviceResult:
    """Result left on the device; valid until the next align call on the index."""

    def __init__(self, r: _DeviceResult):
        self.n_reads = int(r.n_reads)
        self.n_hits = int(r.n_hits)
        self._r = r

    def tensors(self):
        """(total[u64 n], offsets[u64 n+1], hits[u8 8*n_hits]) as torch CUDA tensors (views)."""
        import torch
        t = torch.as_tensor(_CudaArray(self._r.total, (self.n_reads,), "<u8"), device="cuda")
        o = torch.as_tensor(_CudaArray(self._r.offsets, (self.n_reads + 1,), "<u8"), device="cuda")
        h = torch.as_tensor(_CudaArray(self._r.hits, (8 * self.n_hits,), "|u1"), device="cuda")
        return t, o, h


class Index:
    """A resident FM index on one GPU (mica_index)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        self._inflight = {}   # ticket -> the host arrays the library still reads

    @classmethod
    def build(cls, genome_acgt, kmer_q: int = 12, sa_sample: int = 16, device: int = 0,
              lower_bounds: bool = True, full_sa: bool = True) -> "Index":
        """Index of `genome_acgt` (ACGT bytes, a uint8 array of them, or a
        Reference, whose text is passed without a copy)."""
        if isinstance(genome_acgt, Reference):
            ptr, n = genome_acgt._text_ptr()
        else:
            g = _acgt(genome_acgt)
            ptr, n = (_ptr(g) if g.size else None), g.size
        p = IndexParams(kmer_q, sa_sample, int(bool(lower_bounds)), int(bool(full_sa)))
        h = ctypes.c_void_p()
        _check(_lib.mica_index_build_resident(ptr, n, ctypes.byref(p), device, ctypes.byref(h)),
               "mica_index_build_resident")
        return cls(h.value)

    @classmethod
    def load(cls, path: str, device: int = 0) -> "Index":
        h = ctypes.c_void_p()
        _check(_lib.mica_index_load(os.fsencode(path), device, ctypes.byref(h)), "mica_index_load")
        return cls(h.value)

    def save(self, path: str):
        _check(_lib.mica_index_save(self._h, os.fsencode(path)), "mica_index_save")

    def free(self):
        if self._h:
            _lib.mica_index_free(self._h)   # waits for batches still in flight
            self._h = None
            self._inflight.clear()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        i = IndexInfo()
        _check(_lib.mica_index_get_info(self._h, ctypes.byref(i)), "mica_index_get_info")
        d = {name: getattr(i, name) for name, _ in IndexInfo._fields_}
        d["C"] = list(i.C)
        return d

    def set_tuning(self, shape: int = -1, plain_block: int = 0, plain_budget: int = 0, plain_block_len=(0, 0, 0, 0),
                   prefetch: int = -1, bidir_budget: int = 0, bidir_verify: int = 0, bidir_shape: int = -1):
        t = Tuning(shape, plain_block, plain_budget, (ctypes.c_uint32 * 4)(*plain_block_len), prefetch, bidir_budget,
                   bidir_verify, bidir_shape)
        _check(_lib.mica_set_tuning(self._h, ctypes.byref(t)), "mica_set_tuning")

    def autotune(self, batch, hit_cap: int = 1000, repeats: int = 2, cache: str | None = None) -> dict:
        """Pick the fastest launch shapes on `batch` (or reuse a cached choice)."""
        words = np.ascontiguousarray(batch.words, dtype=np.uint32)
        off = np.ascontiguousarray(batch.word_off, dtype=np.uint64)
        lens = np.ascontiguousarray(batch.lengths, dtype=np.uint16)
        k = np.ascontiguousarray(batch.k, dtype=np.uint8)
        classes = 0
        for c, (lo, hi) in enumerate(((1, 64), (65, 128), (129, 192), (193, 256))):
            if np.any((lens >= lo) & (lens <= hi)):
                classes |= 1 << c
        kmax = int(k.max()) if k.size else 0
        t = Tuning()
        if cache and _lib.mica_tuning_cache_lookup(os.fsencode(cache), self._h, classes, kmax, ctypes.byref(t)) == 0:
            _check(_lib.mica_set_tuning(self._h, ctypes.byref(t)), "mica_set_tuning")
            return self.tuning()
        _check(_lib.mica_autotune(self._h, _ptr(words), _ptr(off), _ptr(lens), _ptr(k), lens.size, hit_cap, repeats,
                                  ctypes.byref(t)), "mica_autotune")
        if cache:
            _check(_lib.mica_tuning_cache_store(os.fsencode(cache), self._h, classes, kmax, ctypes.byref(t)),
                   "mica_tuning_cache_store")
        return self.tuning()

    def set_wait_limits(self, idle_rounds: int = 0, ring_spins: int = 0):
        """Bounds of the persistent kernel's device waits (0 = defaults); see mica_set_wait_limits."""
        _check(_lib.mica_set_wait_limits(self._h, idle_rounds, ring_spins), "mica_set_wait_limits")

    def tuning(self) -> dict:
        t = Tuning()
        _check(_lib.mica_get_tuning(self._h, ctypes.byref(t)), "mica_get_tuning")
        return {"shape": t.shape, "plain_block": t.plain_block, "plain_budget": t.plain_budget,
                "plain_block_len": list(t.plain_block_len), "prefetch": t.prefetch, "bidir_budget": t.bidir_budget,
                "bidir_verify": t.bidir_verify, "bidir_shape": t.bidir_shape}

    def stats(self) -> dict:
        s = Stats()
        _check(_lib.mica_get_stats(self._h, ctypes.byref(s)), "mica_get_stats")
        return s.as_dict()

    @staticmethod
    def _params(hit_cap, kernel, stream, prune=True, report="all"):
        return AlignParams(hit_cap, KERNELS[kernel] if isinstance(kernel, str) else int(kernel),
                           _stream_handle(stream), int(bool(prune)),
                           REPORTS[report] if isinstance(report, str) else int(report))

    @staticmethod
    def _host_batch(what, words, word_off, lengths, k):
        words = np.ascontiguousarray(words, dtype=np.uint32)
        word_off = np.ascontiguousarray(word_off, dtype=np.uint64)
        lengths = np.ascontiguousarray(lengths, dtype=np.uint16)
        k = np.ascontiguousarray(k, dtype=np.uint8)
        n = lengths.size
        # the library reads word_off[n] words, n + 1 offsets and n budgets from these buffers
        if word_off.size != n + 1 or k.size != n or int(word_off[-1]) > words.size:
            raise MicaError(MICA_EINVAL, f"{what}: {n} lengths need {n + 1} word offsets (got "
                                         f"{word_off.size}), {n} budgets (got {k.size}) and the words the "
                                         f"last offset names (got {words.size})")
        return words, word_off, lengths, k, n

    def align(self, words, word_off, lengths, k, hit_cap: int = 1000, kernel="bidirectional",
              stream=None, prune: bool = True, report="all") -> Result:
        """mica_align_batch on host arrays (copies in, searches, copies out)."""
        words, word_off, lengths, k, n = self._host_batch("mica_align_batch", words, word_off, lengths, k)
        p = self._params(hit_cap, kernel, stream, prune, report)
        out = ctypes.POINTER(_Result)()
        _check(_lib.mica_align_batch(self._h, _ptr(words) if words.size else None, _ptr(word_off),
                                     _ptr(lengths) if n else None, _ptr(k) if n else None, n,
                                     ctypes.byref(p), ctypes.byref(out)), "mica_align_batch")
        return _take_result(out)

    def submit(self, words, word_off, lengths, k, hit_cap: int = 1000, kernel="bidirectional",
               prune: bool = True, report="all") -> int:
        """mica_align_submit: stage a host batch on a free pipeline slot and
        queue its search; returns the ticket for collect().  The arrays are
        kept alive here until the batch is collected."""
        words, word_off, lengths, k, n = self._host_batch("mica_align_submit", words, word_off, lengths, k)
        p = self._params(hit_cap, kernel, None, prune, report)
        t = ctypes.c_uint64()
        _check(_lib.mica_align_submit(self._h, _ptr(words) if words.size else None, _ptr(word_off),
                                      _ptr(lengths) if n else None, _ptr(k) if n else None, n,
                                      ctypes.byref(p), ctypes.byref(t)), "mica_align_submit")
        self._inflight[t.value] = (words, word_off, lengths, k)
        return t.value

    def collect(self, ticket: int) -> Result:
        """mica_align_collect: wait for a submitted batch and return its result."""
        out = ctypes.POINTER(_Result)()
        rc = _lib.mica_align_collect(self._h, ticket, ctypes.byref(out))
        if rc != MICA_ENOTFOUND:
            self._inflight.pop(ticket, None)   # the library is done with the batch's host arrays
        _check(rc, "mica_align_collect")
        return _take_result(out)

    def submit_batch(self, batch, **kw) -> int:
        """submit() on any object with words/word_off/lengths/k arrays."""
        return self.submit(batch.words, batch.word_off, batch.lengths, batch.k, **kw)

    def align_batch(self, batch, **kw) -> Result:
        """align() on any object with words/word_off/lengths/k arrays."""
        return self.align(batch.words, batch.word_off, batch.lengths, batch.k, **kw)

    def align_device(self, d_words, d_word_off, d_lengths, d_k, n_reads: int, hit_cap: int = 1000,
                     kernel="bidirectional", stream=None, prune: bool = True, report="all") -> DeviceResult:
        """mica_align_device on device pointers (ints) or torch CUDA tensors."""
        ptr = lambda x: x if isinstance(x, int) else x.data_ptr()
        p = self._params(hit_cap, kernel, stream, prune, report)
        r = _DeviceResult()
        _check(_lib.mica_align_device(self._h, ctypes.c_void_p(ptr(d_words)), ctypes.c_void_p(ptr(d_word_off)),
                                      ctypes.c_void_p(ptr(d_lengths)), ctypes.c_void_p(ptr(d_k)), n_reads,
                                      ctypes.byref(p), ctypes.byref(r)), "mica_align_device")
        return DeviceResult(r)

    # ---- parity probes ----
    def debug_occ(self, rows) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.uint64)
        out = np.empty((rows.size, 4), dtype=np.uint32)
        _check(_lib.mica_debug_occ(self._h, _ptr(rows), rows.size, _ptr(out)), "mica_debug_occ")
        return out

    def debug_locate(self, rows) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.uint64)
        out = np.empty(rows.size, dtype=np.uint32)
        _check(_lib.mica_debug_locate(self._h, _ptr(rows), rows.size, _ptr(out)), "mica_debug_locate")
        return out

    def debug_full_sa(self, which: str, first: int = 0, n: int | None = None) -> np.ndarray:
        """Entries of the resident whole suffix array ("sa"), its inverse ("isa")
        or the 2-bit text words ("text") (mica_debug_full_sa)."""
        w = {"sa": 0, "isa": 1, "text": 2}[which]
        info = self.info()
        length = info["rows"] if w < 2 else (info["full_sa_bytes"] - 8 * info["rows"]) // 4
        if n is None:
            n = length - first
        out = np.empty(n, dtype=np.uint32)
        _check(_lib.mica_debug_full_sa(self._h, w, first, n, _ptr(out) if n else None), "mica_debug_full_sa")
        return out

    def debug_lower_bounds(self, batch) -> np.ndarray:
        """Lower-bound words of the 2n (read, strand) tasks (mica_debug_lower_bounds)."""
        words = np.ascontiguousarray(batch.words, dtype=np.uint32)
        off = np.ascontiguousarray(batch.word_off, dtype=np.uint64)
        lens = np.ascontiguousarray(batch.lengths, dtype=np.uint16)
        k = np.ascontiguousarray(batch.k, dtype=np.uint8)
        out = np.empty(2 * lens.size, dtype=np.uint64)
        _check(_lib.mica_debug_lower_bounds(self._h, _ptr(words) if words.size else None, _ptr(off),
                                            _ptr(lens) if lens.size else None, _ptr(k) if k.size else None,
                                            lens.size, _ptr(out) if out.size else None), "mica_debug_lower_bounds")
        return out

    def debug_table_interval(self, which: str, codes, length: int) -> np.ndarray:
        """[l, r) of each length-mer code from one seed table: "fwd", "rev" (the
        q-mer tables of G$ and G~$), "long_fwd", "long_rev" (the longer ones)."""
        w = {"fwd": 0, "rev": 1, "long_fwd": 2, "long_rev": 3}[which]
        codes = np.ascontiguousarray(codes, dtype=np.uint32)
        out = np.empty((codes.size, 2), dtype=np.uint32)
        _check(_lib.mica_debug_table_interval(self._h, w, _ptr(codes) if codes.size else None, length, codes.size,
                                              _ptr(out) if codes.size else None), "mica_debug_table_interval")
        return out

    def debug_seed_interval(self, codes, length: int) -> np.ndarray:
        """[l, r) of each length-mer code from the q-mer table (GPU seed step)."""
        codes = np.ascontiguousarray(codes, dtype=np.uint32)
        out = np.empty((codes.size, 2), dtype=np.uint32)
        _check(_lib.mica_debug_seed_interval(self._h, _ptr(codes), length, codes.size, _ptr(out)),
               "mica_debug_seed_interval")
        return out


class Server:
    """Continuous-batching request loop over a resident index (mica_server_*)."""

    def __init__(self, index: Index, max_device_bytes: int = 0, max_tick_reads: int = 0, hit_cap: int = 1000,
                 kernel="bidirectional", workers: int = 2, start_paused: bool = False, chunk_reads: int = 0):
        p = ServerParams()
        _lib.mica_server_params_default(ctypes.byref(p))
        p.max_device_bytes = max_device_bytes
        p.max_tick_reads = max_tick_reads
        p.chunk_reads = chunk_reads
        p.hit_cap = hit_cap
        p.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        p.workers = workers
        p.start_paused = int(start_paused)
        self.index = index
        h = ctypes.c_void_p()
        _check(_lib.mica_server_start(index._h, ctypes.byref(p), ctypes.byref(h)), "mica_server_start")
        self._h = h

    @staticmethod
    def workspace_bytes(index: Index, n_reads: int, n_words: int) -> int:
        """Device bytes one worker needs for a tick of n_reads reads (mica_server_workspace_bytes)."""
        b = ctypes.c_uint64()
        _check(_lib.mica_server_workspace_bytes(index._h, n_reads, n_words, ctypes.byref(b)),
               "mica_server_workspace_bytes")
        return int(b.value)

    def submit(self, words, word_off, lengths, k) -> int:
        words = np.ascontiguousarray(words, dtype=np.uint32)
        word_off = np.ascontiguousarray(word_off, dtype=np.uint64)
        lengths = np.ascontiguousarray(lengths, dtype=np.uint16)
        k = np.ascontiguousarray(k, dtype=np.uint8)
        rid = ctypes.c_uint64()
        n = lengths.size
        _check(_lib.mica_server_submit(self._h, _ptr(words) if words.size else None, _ptr(word_off),
                                       _ptr(lengths) if n else None, _ptr(k) if n else None, n,
                                       ctypes.byref(rid)), "mica_server_submit")
        return int(rid.value)

    def submit_batch(self, batch) -> int:
        return self.submit(batch.words, batch.word_off, batch.lengths, batch.k)

    def poll(self, rid: int):
        """(Result, latency_ms) once done, None while queued or running."""
        out = ctypes.POINTER(_Result)()
        lat = ctypes.c_double()
        rc = _lib.mica_server_poll(self._h, rid, ctypes.byref(out), ctypes.byref(lat))
        if rc == MICA_EBUSY:
            return None
        _check(rc, "mica_server_poll")
        return _take_result(out), lat.value

    def wait(self, rid: int, timeout_ms: int = 600_000):
        out = ctypes.POINTER(_Result)()
        lat = ctypes.c_double()
        _check(_lib.mica_server_wait(self._h, rid, timeout_ms, ctypes.byref(out), ctypes.byref(lat)),
               "mica_server_wait")
        return _take_result(out), lat.value

    def cancel(self, rid: int) -> int:
        return int(_lib.mica_server_cancel(self._h, rid))

    def resume(self):
        _lib.mica_server_resume(self._h)

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.mica_server_get_stats(self._h, ctypes.byref(st)), "mica_server_get_stats")
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def stop(self):
        if self._h:
            _lib.mica_server_stop(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.stop()


NOALLOC_MAX_COUNTS = 1 << 24


def offsets_noalloc(d_counts, n: int, d_offsets, stream=None) -> None:
    """mica_offsets_noalloc: CSR offsets from per-read counts (device
    pointers or torch CUDA tensors), without allocating device memory.

    Tensors must be 8-byte integer CUDA tensors on the current device with at
    least n (counts) and n + 1 (offsets) elements; anything else raises
    MicaError(MICA_EINVAL) before the call.  With tensors and no stream, the
    call runs on torch's current stream, which is where they were produced;
    with raw pointers and no stream, on the legacy default stream."""
    tensors = [x for x in (d_counts, d_offsets) if not isinstance(x, int)]
    if tensors:
        import torch
        dev = torch.cuda.current_device()
        for x, need, what in ((d_counts, n, "counts"), (d_offsets, n + 1, "offsets")):
            if isinstance(x, int):
                continue
            if not (x.is_cuda and x.device.index == dev and x.element_size() == 8 and
                    not x.dtype.is_floating_point and x.is_contiguous() and x.numel() >= need):
                raise MicaError(MICA_EINVAL, f"offsets_noalloc: {what} must be a contiguous 8-byte integer "
                                             f"CUDA tensor on device {dev} with at least {need} elements")
        if stream is None:
            stream = torch.cuda.current_stream()
    ptr = lambda x: x if isinstance(x, int) else x.data_ptr()
    _check(_lib.mica_offsets_noalloc(ctypes.c_void_p(ptr(d_counts)), n, ctypes.c_void_p(ptr(d_offsets)),
                                     _stream_handle(stream)), "mica_offsets_noalloc")


PAIR_DTYPE = np.dtype([("n_concordant", np.uint32), ("n_best", np.uint32), ("pos_plus", np.uint32),
                       ("pos_minus", np.uint32), ("plus_mate", np.uint8), ("mm", np.uint8), ("pad", np.uint16)])


def pair_batch(result, lengths, insert_min: int, insert_max: int, device: int = 0) -> np.ndarray:
    """mica_pair_batch: mate pairing of a host Result whose reads 2i, 2i+1 are
    the mates of pair i; returns a PAIR_DTYPE array, one row per pair."""
    off = np.ascontiguousarray(result.offsets, dtype=np.uint64)
    hits = np.ascontiguousarray(result.hits)
    lens = np.ascontiguousarray(lengths, dtype=np.uint16)
    n_pairs = (off.size - 1) // 2
    out = np.zeros(n_pairs, dtype=PAIR_DTYPE)
    _check(_lib.mica_pair_batch(device, _ptr(off), _ptr(hits) if hits.size else None, _ptr(lens) if lens.size else None,
                                n_pairs, insert_min, insert_max, _ptr(out) if n_pairs else None), "mica_pair_batch")
    return out


def pair_device(d_offsets, d_hits, d_lengths, n_pairs: int, insert_min: int, insert_max: int, d_out,
                stream=None) -> None:
    """mica_pair_device on device pointers (ints) or torch CUDA tensors."""
    ptr = lambda x: x if isinstance(x, int) else x.data_ptr()
    _check(_lib.mica_pair_device(ctypes.c_void_p(ptr(d_offsets)), ctypes.c_void_p(ptr(d_hits)),
                                 ctypes.c_void_p(ptr(d_lengths)), n_pairs, insert_min, insert_max,
                                 ctypes.c_void_p(ptr(d_out)), _stream_handle(stream)), "mica_pair_device")


class ReferenceInfo(ctypes.Structure):
    _fields_ = [("length", ctypes.c_uint64), ("n_contigs", ctypes.c_uint64), ("n_ambiguous_runs", ctypes.c_uint64),
                ("ambiguous_bases", ctypes.c_uint64)]


class SamParams(ctypes.Structure):
    _fields_ = [("qname_prefix", ctypes.c_char_p), ("secondary", ctypes.c_uint32), ("command_line", ctypes.c_char_p),
                ("threads", ctypes.c_uint32)]


class Reference:
    """Named contigs concatenated into the index's text G (mica_reference):
    ambiguous bytes replaced by a coordinate-derived base and recorded as
    runs.  Host-only; build the index from :meth:`text`."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @classmethod
    def create(cls, sequence, contig_lengths, names=None) -> "Reference":
        seq = _acgt(sequence)
        cl = np.ascontiguousarray(contig_lengths, dtype=np.uint64)
        arr = None
        if names is not None:
            arr = (ctypes.c_char_p * len(names))(*[n.encode() for n in names])
        out = ctypes.c_void_p()
        _check(_lib.mica_reference_create(_ptr(seq) if seq.size else None, seq.size, _ptr(cl) if cl.size else None,
                                          arr, cl.size, ctypes.byref(out)), "mica_reference_create")
        return cls(out.value)

    @classmethod
    def from_fasta(cls, path: str) -> "Reference":
        out = ctypes.c_void_p()
        _check(_lib.mica_reference_read_fasta(path.encode(), ctypes.byref(out)), "mica_reference_read_fasta")
        return cls(out.value)

    @classmethod
    def load(cls, path: str) -> "Reference":
        out = ctypes.c_void_p()
        _check(_lib.mica_reference_load(path.encode(), ctypes.byref(out)), "mica_reference_load")
        return cls(out.value)

    def save(self, path: str):
        _check(_lib.mica_reference_save(self._h, path.encode()), "mica_reference_save")

    def free(self):
        if self._h:
            _lib.mica_reference_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        i = ReferenceInfo()
        _check(_lib.mica_reference_get_info(self._h, ctypes.byref(i)), "mica_reference_get_info")
        return {f: int(getattr(i, f)) for f, _ in ReferenceInfo._fields_}

    def _text_ptr(self):
        p, n = ctypes.c_void_p(), ctypes.c_uint64()
        _check(_lib.mica_reference_text(self._h, ctypes.byref(p), ctypes.byref(n)), "mica_reference_text")
        return p, int(n.value)

    def text(self) -> bytes:
        """G as 'ACGT' bytes (a copy); Index.build(reference) needs no copy."""
        p, n = self._text_ptr()
        return ctypes.string_at(p.value, n) if n else b""

    def contigs(self) -> list:
        """[(name, start, length)] in order."""
        out = []
        for i in range(self.info()["n_contigs"]):
            name, st, ln = ctypes.c_char_p(), ctypes.c_uint64(), ctypes.c_uint64()
            _check(_lib.mica_reference_contig(self._h, i, ctypes.byref(name), ctypes.byref(st), ctypes.byref(ln)),
                   "mica_reference_contig")
            out.append((name.value.decode(), int(st.value), int(ln.value)))
        return out

    def ambiguous_runs(self) -> np.ndarray:
        """(start, length) of every maximal run of ambiguous coordinates of G."""
        n = self.info()["n_ambiguous_runs"]
        out = np.zeros((n, 2), dtype=np.uint64)
        st, ln = ctypes.c_uint64(), ctypes.c_uint64()
        for j in range(n):
            _check(_lib.mica_reference_ambiguous_run(self._h, j, ctypes.byref(st), ctypes.byref(ln)),
                   "mica_reference_ambiguous_run")
            out[j] = (st.value, ln.value)
        return out

    def locate(self, pos, span):
        """(contig int32, local uint32) of windows [pos, pos + span) of G;
        contig -1 when the window is not a placement on the reference."""
        pos = np.ascontiguousarray(pos, dtype=np.uint32)
        span = np.ascontiguousarray(np.broadcast_to(span, pos.shape), dtype=np.uint16)
        contig = np.empty(pos.size, dtype=np.int32)
        local = np.empty(pos.size, dtype=np.uint32)
        if pos.size:
            _check(_lib.mica_reference_locate(self._h, _ptr(pos), _ptr(span), pos.size, _ptr(contig), _ptr(local)),
                   "mica_reference_locate")
        return contig, local

    def filter(self, result, lengths):
        """A copy of a host Result without the hits that are not placements on
        the reference (mica_reference_filter); returns (Result, n_dropped)."""
        total = np.array(result.total, dtype=np.uint64)
        off = np.array(result.offsets, dtype=np.uint64)
        hits = np.array(result.hits, dtype=HIT_DTYPE)
        lens = np.ascontiguousarray(lengths, dtype=np.uint16)
        dropped = ctypes.c_uint64()
        n = total.size
        _check(_lib.mica_reference_filter(self._h, _ptr(lens) if n else None, n, _ptr(total) if n else None,
                                          _ptr(off), _ptr(hits) if hits.size else None, ctypes.byref(dropped)),
               "mica_reference_filter")
        return Result(total, off, hits[:int(off[-1])].copy()), int(dropped.value)


class ReadBatchView(ctypes.Structure):
    _fields_ = [("n_reads", ctypes.c_uint64), ("packed_reads", ctypes.c_void_p), ("word_offsets", ctypes.c_void_p),
                ("lengths", ctypes.c_void_p), ("k", ctypes.c_void_p), ("n_ambiguous_reads", ctypes.c_uint64),
                ("paired", ctypes.c_uint32)]


def _copy_array(ptr, n: int, dtype) -> np.ndarray:
    out = np.empty(n, dtype=dtype)
    if n:
        ctypes.memmove(out.ctypes.data, ptr, n * out.itemsize)
    return out


class FastqBatch:
    """Reads of one mica_fastq_read call (mica_read_batch): words, word_off,
    lengths and k as numpy copies (so `Index.align_batch(batch)` works), plus
    names, qualities and the offsets of ambiguous bases."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        v = ReadBatchView()
        _check(_lib.mica_read_batch_get_view(self._h, ctypes.byref(v)), "mica_read_batch_get_view")
        n = int(v.n_reads)
        self.word_off = _copy_array(v.word_offsets, n + 1, np.uint64)
        self.words = _copy_array(v.packed_reads, int(self.word_off[-1]), np.uint32)
        self.lengths = _copy_array(v.lengths, n, np.uint16)
        self.k = _copy_array(v.k, n, np.uint8)
        self.n_ambiguous_reads = int(v.n_ambiguous_reads)
        self.paired = bool(v.paired)

    @property
    def n(self) -> int:
        return int(self.lengths.size)

    def read(self, i: int) -> np.ndarray:
        """Base codes of read i as searched (ambiguous bases hold their stand-ins)."""
        m = int(self.lengths[i])
        w = self.words[int(self.word_off[i]):int(self.word_off[i + 1])]
        return ((w[:, None] >> (2 * np.arange(16, dtype=np.uint32))[None, :]) & 3).astype(np.uint8).reshape(-1)[:m]

    def record(self, i: int):
        """(name, qualities, ambiguous offsets) of read i."""
        name, qual, amb, na = ctypes.c_char_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_uint32()
        _check(_lib.mica_read_batch_read(self._h, i, ctypes.byref(name), ctypes.byref(qual), ctypes.byref(amb),
                                         ctypes.byref(na)), "mica_read_batch_read")
        m = int(self.lengths[i])
        return (name.value.decode(), ctypes.string_at(qual.value, m).decode(),
                _copy_array(amb.value, int(na.value), np.uint16))

    def filter_n(self, reference: "Reference", result):
        """A copy of this batch's host Result with ambiguous read bases counted
        as substitutions (mica_read_batch_filter_n); returns (Result, n_dropped)."""
        total = np.array(result.total, dtype=np.uint64)
        off = np.array(result.offsets, dtype=np.uint64)
        hits = np.array(result.hits, dtype=HIT_DTYPE)
        dropped = ctypes.c_uint64()
        _check(_lib.mica_read_batch_filter_n(self._h, reference._h, _ptr(total) if total.size else None, _ptr(off),
                                             _ptr(hits) if hits.size else None, ctypes.byref(dropped)),
               "mica_read_batch_filter_n")
        return Result(total, off, hits[:int(off[-1])].copy()), int(dropped.value)

    def free(self):
        if self._h:
            _lib.mica_read_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class FastqReader:
    """Batches of reads from one FASTQ file, or two files of mates (mica_fastq)."""

    def __init__(self, path1: str, path2: str | None = None):
        out = ctypes.c_void_p()
        _check(_lib.mica_fastq_open(path1.encode(), path2.encode() if path2 else None, ctypes.byref(out)),
               "mica_fastq_open")
        self._h = ctypes.c_void_p(out.value)

    def read(self, max_reads: int, k: int = 2) -> FastqBatch:
        """The next batch (0 reads at the end)."""
        out = ctypes.c_void_p()
        _check(_lib.mica_fastq_read(self._h, max_reads, k, ctypes.byref(out)), "mica_fastq_read")
        return FastqBatch(out.value)

    def batches(self, max_reads: int, k: int = 2):
        while True:
            b = self.read(max_reads, k)
            if b.n == 0:
                return
            yield b

    def close(self):
        if self._h:
            _lib.mica_fastq_close(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SamWriter:
    """SAM output of results against a Reference (mica_sam_*).  Keep the
    Reference alive until close()."""

    def __init__(self, path: str, reference: Reference, qname_prefix: str = "r", secondary: bool = False,
                 command_line: str | None = None, threads: int = 0):
        self._ref = reference
        p = SamParams(qname_prefix.encode(), int(secondary), command_line.encode() if command_line else None,
                      threads)
        out = ctypes.c_void_p()
        _check(_lib.mica_sam_open(path.encode(), reference._h, ctypes.byref(p), ctypes.byref(out)), "mica_sam_open")
        self._h = ctypes.c_void_p(out.value)

    def write(self, batch, result, pairs=None):
        """Records of one batch (a ReadBatch-like object with words, word_off,
        lengths) and its host Result; pairs: PAIR_DTYPE rows from pair_batch
        when reads 2i, 2i+1 are mates."""
        words = np.ascontiguousarray(batch.words, dtype=np.uint32)
        woff = np.ascontiguousarray(batch.word_off, dtype=np.uint64)
        lens = np.ascontiguousarray(batch.lengths, dtype=np.uint16)
        total = np.ascontiguousarray(result.total, dtype=np.uint64)
        off = np.ascontiguousarray(result.offsets, dtype=np.uint64)
        hits = np.ascontiguousarray(result.hits, dtype=HIT_DTYPE)
        n = lens.size
        pr = None if pairs is None else np.ascontiguousarray(pairs, dtype=PAIR_DTYPE)
        if n == 0:
            return
        _check(_lib.mica_sam_write(self._h, _ptr(words) if words.size else None, _ptr(woff), _ptr(lens), n,
                                   _ptr(total), _ptr(off), _ptr(hits) if hits.size else None,
                                   _ptr(pr) if pr is not None and pr.size else None), "mica_sam_write")

    def write_batch(self, batch: FastqBatch, result, pairs=None):
        """Records of a FastqBatch and its host Result (names, qualities, N)."""
        if batch.n == 0:
            return
        total = np.ascontiguousarray(result.total, dtype=np.uint64)
        off = np.ascontiguousarray(result.offsets, dtype=np.uint64)
        hits = np.ascontiguousarray(result.hits, dtype=HIT_DTYPE)
        pr = None if pairs is None else np.ascontiguousarray(pairs, dtype=PAIR_DTYPE)
        _check(_lib.mica_sam_write_batch(self._h, batch._h, _ptr(total), _ptr(off), _ptr(hits) if hits.size else None,
                                         _ptr(pr) if pr is not None and pr.size else None), "mica_sam_write_batch")

    def close(self):
        if self._h:
            h, self._h = self._h, None
            _check(_lib.mica_sam_close(h), "mica_sam_close")

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gather_ceiling(buffer_bytes: int, load_bytes: int = 32, loads: int = 1 << 28, repeats: int = 3,
                   device: int = 0) -> dict:
    """mica_gather_ceiling: GB/s of independent random `load_bytes` loads
    from a device buffer of `buffer_bytes` (the search's access pattern)."""
    gbs, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.mica_gather_ceiling(device, buffer_bytes, load_bytes, loads, repeats, ctypes.byref(gbs),
                                    ctypes.byref(ms)), "mica_gather_ceiling")
    return {"gbs": gbs.value, "ms": ms.value, "buffer_bytes": buffer_bytes, "load_bytes": load_bytes}


def debug_suffix_array(genome_acgt, device: int = 0) -> np.ndarray:
    """Suffix array of G$ built on the GPU (mica_debug_suffix_array)."""
    g = _acgt(genome_acgt)
    sa = np.empty(g.size + 1, dtype=np.uint32)
    _check(_lib.mica_debug_suffix_array(_ptr(g) if g.size else None, g.size, device, _ptr(sa)),
           "mica_debug_suffix_array")
    return sa


def exported_symbols() -> list:
    return sorted(SIGNATURES)
