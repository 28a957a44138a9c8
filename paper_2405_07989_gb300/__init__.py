"""GB300 factorization sets: Python binding of the C ABI in include/fs.h.

The binding only marshals arguments: every step of the computation runs in
the CUDA kernels of ``libfs.so``.  There is no CPU fallback; if the library is
missing or no GPU is usable, calls raise :class:`FsError`.

Device buffers are torch CUDA tensors (their ``data_ptr()`` is passed); the
stream defaults to torch's current stream.  Function names follow the C ABI.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfs.so")
MAX_D = 16

FS_OK, FS_E_INVAL, FS_E_OVERFLOW, FS_E_CAPACITY = 0, 1, 2, 3
FS_E_NOMEM, FS_E_CUDA, FS_E_TIMEOUT, FS_E_NOTIMPL = 4, 5, 6, 7
METHOD_AUTO, METHOD_PLAIN, METHOD_PAIR, METHOD_TRIPLE, METHOD_QUAD = 0, 1, 2, 3, 4
WALK_AUTO, WALK_PACKED, WALK_LANES = 0, 1, 2

_lock = threading.Lock()
_lib = None


class FsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


class fs_config(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("keep_order", ctypes.c_int32),
                ("slices", ctypes.c_int64), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("walk", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class fs_len_summary(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("min_len", ctypes.c_uint32),
                ("max_len", ctypes.c_uint32)]


class fs_predicate(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32 * MAX_D), ("c", ctypes.c_int64), ("op", ctypes.c_int32),
                ("modulus", ctypes.c_uint32)]


class fs_query(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("gens", ctypes.c_uint32 * MAX_D)]


class fs_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("min_len", ctypes.c_uint32),
                ("max_len", ctypes.c_uint32), ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


BATCH_COUNT, BATCH_LENGTHS = 0, 1
REQ_COUNT, REQ_LENGTHS, REQ_ENUMERATE = 0, 1, 2


class fs_server_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("table_bytes", ctypes.c_uint64),
                ("max_batch", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("window_us", ctypes.c_int32), ("job_streams", ctypes.c_int32),
                ("hist_max_leaves", ctypes.c_uint64), ("direct_leaves", ctypes.c_uint64)]


class fs_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("gens", ctypes.c_uint32 * MAX_D),
                ("op", ctypes.c_int32), ("elem_bytes", ctypes.c_int32),
                ("keep_order", ctypes.c_int32), ("hist", ctypes.c_int32)]


class fs_response(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("op", ctypes.c_int32),
                ("count", ctypes.c_uint64), ("min_len", ctypes.c_uint32),
                ("max_len", ctypes.c_uint32), ("rows", ctypes.c_void_p),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_counted", ctypes.c_double), ("t_job", ctypes.c_double),
                ("t_done", ctypes.c_double)]

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_vp = ctypes.c_void_p
_cfgp = ctypes.POINTER(fs_config)

# name -> (restype, argtypes): every entry point declared in include/fs.h
SIGNATURES = {
    "fs_config_default": (None, [_cfgp]),
    "fs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fs_version": (ctypes.c_int, []),
    "fs_last_error": (ctypes.c_char_p, []),
    "fs_count": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _u64p, _vp]),
    "fs_length_stats": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int,
                                       ctypes.POINTER(fs_len_summary), _vp, _vp]),
    "fs_any": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int,
                              ctypes.POINTER(fs_predicate), ctypes.POINTER(ctypes.c_int), _vp]),
    "fs_enumerate": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _vp, ctypes.c_uint64,
                                    ctypes.c_int, _u64p, _vp]),
    "fs_count_ex": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp, _u64p, _vp]),
    "fs_length_stats_async": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp, _vp, _vp,
                                             _vp]),
    "fs_length_stats_ex": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp,
                                          ctypes.POINTER(fs_len_summary), _vp, _vp]),
    "fs_any_ex": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp,
                                 ctypes.POINTER(fs_predicate), ctypes.POINTER(ctypes.c_int), _vp]),
    "fs_enumerate_ex": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp, _vp,
                                       ctypes.c_uint64, ctypes.c_int, _u64p, _vp]),
    "fs_count_async": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp, _vp, _vp]),
    "fs_enumerate_async": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp, _vp,
                                          ctypes.c_uint64, ctypes.c_int, _vp, _vp]),
    "fs_cursor_create": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp, ctypes.c_int,
                                        _vp, ctypes.POINTER(ctypes.c_void_p)]),
    "fs_cursor_count": (ctypes.c_int, [_vp, _u64p]),
    "fs_cursor_tell": (ctypes.c_int, [_vp, _u64p]),
    "fs_cursor_slices": (ctypes.c_int, [_vp, _u64p]),
    "fs_cursor_seek": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "fs_cursor_next": (ctypes.c_int, [_vp, _vp, ctypes.c_uint64, _u64p, _vp]),
    "fs_cursor_destroy": (ctypes.c_int, [_vp]),
    "fs_enumerate_host": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp, _vp,
                                         ctypes.c_uint64, ctypes.c_int, _u64p, _vp]),
    "fs_plan": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp, ctypes.c_int64,
                               _i32p, _i32p, _u64p]),
    "fs_slice_counts": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _cfgp,
                                       ctypes.c_int64, _u64p, _vp]),
    "fs_count_noalloc": (ctypes.c_int, [ctypes.c_int64, _u32p, ctypes.c_int, _vp, _vp]),
    "fs_alloc_counts": (None, [_u64p, _u64p]),
    "fs_batch_create": (ctypes.c_int, [ctypes.POINTER(fs_query), ctypes.c_int, ctypes.c_int, _cfgp,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "fs_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "fs_batch_load_mode": (ctypes.c_int, [_vp, ctypes.POINTER(fs_query), ctypes.c_int, ctypes.c_int,
                                          _vp]),
    "fs_batch_results": (ctypes.c_int, [_vp, ctypes.POINTER(fs_result), _vp]),
    "fs_batch_destroy": (ctypes.c_int, [_vp]),
    "fs_batch_run": (ctypes.c_int, [ctypes.POINTER(fs_query), ctypes.c_int, ctypes.c_int, _cfgp,
                                    ctypes.POINTER(fs_result), _vp]),
    "fs_batch_autotune": (ctypes.c_int, [ctypes.POINTER(fs_query), ctypes.c_int, ctypes.c_int,
                                         _cfgp, ctypes.POINTER(ctypes.c_double), _vp]),
    "fs_batch_table_bytes": (ctypes.c_int, [ctypes.POINTER(fs_query), ctypes.c_int, ctypes.c_int,
                                            _cfgp, _u64p]),
    "fs_batch_reserve": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, _cfgp,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "fs_batch_load": (ctypes.c_int, [_vp, ctypes.POINTER(fs_query), ctypes.c_int, _vp]),
    "fs_batch_fetch": (ctypes.c_int, [_vp, _vp]),
    "fs_batch_collect": (ctypes.c_int, [_vp, ctypes.POINTER(fs_result)]),
    "fs_reserve": (ctypes.c_int, [ctypes.c_uint64, _vp]),
    "fs_server_create": (ctypes.c_int, [ctypes.POINTER(fs_server_config),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "fs_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(fs_request), _u64p]),
    "fs_server_poll": (ctypes.c_int, [_vp, ctypes.POINTER(fs_response), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "fs_server_release": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "fs_server_destroy": (ctypes.c_int, [_vp]),
    "fs_profile_enable": (None, [ctypes.c_int]),
    "fs_profile_only": (None, [ctypes.c_char_p]),
    "fs_profile_read": (ctypes.c_int, [ctypes.c_char_p, _u64p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_int]),
    "fs_probe_int_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32,
                                         ctypes.POINTER(ctypes.c_double)]),
    "fs_selftest_division": (ctypes.c_int64, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]),
    "fs_selftest_split": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_uint64)]),
}


def status_name(s: int) -> str:
    names = ["FS_OK", "FS_E_INVAL", "FS_E_OVERFLOW", "FS_E_CAPACITY", "FS_E_NOMEM",
             "FS_E_CUDA", "FS_E_TIMEOUT", "FS_E_NOTIMPL"]
    return names[s] if 0 <= s < len(names) else f"FS_E_{s}"


def lib():
    """Load libfs.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import _build
            if _build.stale():
                _build.build()
            if not os.path.exists(LIB_PATH):
                raise FsError(FS_E_CUDA, f"{LIB_PATH} is missing: the CUDA library was not built")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st: int):
    if st != FS_OK:
        raise FsError(st, lib().fs_last_error().decode())


def _gens(gens):
    g = [int(x) for x in gens]
    arr = (ctypes.c_uint32 * max(len(g), 1))(*[x & 0xffffffff for x in g])
    return arr, len(g)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def make_config(method: int = METHOD_AUTO, keep_order: bool = False, slices: int = 0,
                block_threads: int = 0, blocks_per_sm: int = 0, walk: int = 0) -> fs_config:
    return fs_config(int(method), int(bool(keep_order)), int(slices), int(block_threads),
                     int(blocks_per_sm), int(walk), 0)


def _cfgp_of(cfg):
    return ctypes.byref(cfg) if cfg is not None else None


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    return ctypes.c_void_p(t.data_ptr())


def fs_version() -> int:
    return lib().fs_version()


def fs_count(n: int, gens, cfg: fs_config | None = None, stream=None) -> int:
    """|Z(n, gens)| (fs_count_ex)."""
    g, d = _gens(gens)
    out = ctypes.c_uint64(0)
    _check(lib().fs_count_ex(int(n), g, d, _cfgp_of(cfg), ctypes.byref(out), _stream(stream)))
    return int(out.value)


def fs_count_async(n: int, gens, dev_count, cfg: fs_config | None = None, stream=None) -> None:
    """Enqueue the count; dev_count is a CUDA uint64/int64 tensor of >= 1 element."""
    g, d = _gens(gens)
    _check(lib().fs_count_async(int(n), g, d, _cfgp_of(cfg), _ptr(dev_count), _stream(stream)))


def fs_length_stats(n: int, gens, hist=None, cfg: fs_config | None = None, stream=None):
    """(count, min_len, max_len); hist (optional) is a CUDA int64 tensor of
    floor(n / min g) + 1 bins, overwritten with the length histogram."""
    g, d = _gens(gens)
    out = fs_len_summary()
    _check(lib().fs_length_stats_ex(int(n), g, d, _cfgp_of(cfg), ctypes.byref(out), _ptr(hist),
                                    _stream(stream)))
    return int(out.count), int(out.min_len), int(out.max_len)


def fs_length_stats_async(n: int, gens, hist=None, out=None, cfg: fs_config | None = None,
                          stream=None) -> None:
    """Enqueue the length statistics: hist (optional CUDA int64 tensor of
    floor(n / min g) + 1 bins) receives the histogram, out (optional CUDA int64
    tensor of 3) the count, min and max, in stream order."""
    g, d = _gens(gens)
    _check(lib().fs_length_stats_async(int(n), g, d, _cfgp_of(cfg), _ptr(hist), _ptr(out),
                                       _stream(stream)))


def fs_any(n: int, gens, w, c: int, op: int = 0, modulus: int = 0,
           cfg: fs_config | None = None, stream=None) -> bool:
    """True iff some factorization a has sum w_i a_i (==, <=, >= by op) c, or
    sum w_i a_i == c (mod modulus) when modulus > 0."""
    g, d = _gens(gens)
    p = fs_predicate()
    for i, x in enumerate(list(w)[:MAX_D]):
        p.w[i] = int(x)
    p.c = int(c)
    p.op = int(op)
    p.modulus = int(modulus)
    out = ctypes.c_int(0)
    _check(lib().fs_any_ex(int(n), g, d, _cfgp_of(cfg), ctypes.byref(p), ctypes.byref(out),
                           _stream(stream)))
    return bool(out.value)


def fs_enumerate(n: int, gens, out, cap: int | None = None, elem_bytes: int = 4,
                 cfg: fs_config | None = None, stream=None, allow_capacity: bool = False) -> int:
    """Write Z(n, gens) into the CUDA tensor `out` (rows [count][d] of int32 or
    int16); returns |Z|.  cap defaults to the rows `out` holds."""
    g, d = _gens(gens)
    if cap is None:
        cap = out.numel() // max(d, 1) if out is not None else 0
    cnt = ctypes.c_uint64(0)
    st = lib().fs_enumerate_ex(int(n), g, d, _cfgp_of(cfg), _ptr(out), int(cap), int(elem_bytes),
                               ctypes.byref(cnt), _stream(stream))
    if st == FS_E_CAPACITY and allow_capacity:
        return int(cnt.value)
    _check(st)
    return int(cnt.value)


def fs_enumerate_async(n: int, gens, out, cap: int, dev_count, elem_bytes: int = 4,
                       cfg: fs_config | None = None, stream=None) -> None:
    """Enqueue the enumeration into `out`; |Z| lands in dev_count[0]."""
    g, d = _gens(gens)
    _check(lib().fs_enumerate_async(int(n), g, d, _cfgp_of(cfg), _ptr(out), int(cap),
                                    int(elem_bytes), _ptr(dev_count), _stream(stream)))


class Cursor:
    """fs_cursor_*: the ordered rows of Z(n, gens), produced window by window.
    next(out) writes up to out's rows into the CUDA tensor `out` and returns
    how many; count / tell / seek as the C functions."""

    def __init__(self, n: int, gens, elem_bytes: int = 4, cfg: fs_config | None = None,
                 stream=None):
        g, d = _gens(gens)
        self.d = d
        h = ctypes.c_void_p(0)
        _check(lib().fs_cursor_create(int(n), g, d, _cfgp_of(cfg), int(elem_bytes),
                                      _stream(stream), ctypes.byref(h)))
        self._h = h

    def count(self) -> int:
        v = ctypes.c_uint64(0)
        _check(lib().fs_cursor_count(self._h, ctypes.byref(v)))
        return int(v.value)

    def tell(self) -> int:
        v = ctypes.c_uint64(0)
        _check(lib().fs_cursor_tell(self._h, ctypes.byref(v)))
        return int(v.value)

    def slices(self) -> int:
        v = ctypes.c_uint64(0)
        _check(lib().fs_cursor_slices(self._h, ctypes.byref(v)))
        return int(v.value)

    def seek(self, row: int) -> None:
        _check(lib().fs_cursor_seek(self._h, int(row)))

    def next(self, out, cap: int | None = None, stream=None) -> int:
        if cap is None:
            cap = out.numel() // max(self.d, 1)
        m = ctypes.c_uint64(0)
        _check(lib().fs_cursor_next(self._h, _ptr(out), int(cap), ctypes.byref(m),
                                    _stream(stream)))
        return int(m.value)

    def close(self):
        if self._h:
            lib().fs_cursor_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fs_enumerate_host(n: int, gens, out, cap: int | None = None, elem_bytes: int = 4,
                      cfg: fs_config | None = None, stream=None,
                      allow_capacity: bool = False) -> int:
    """Write Z(n, gens) into the HOST tensor `out` (pinned for full speed),
    streamed through device staging buffers; returns |Z|."""
    g, d = _gens(gens)
    if cap is None:
        cap = out.numel() // max(d, 1) if out is not None else 0
    cnt = ctypes.c_uint64(0)
    st = lib().fs_enumerate_host(int(n), g, d, _cfgp_of(cfg), _ptr(out), int(cap),
                                 int(elem_bytes), ctypes.byref(cnt), _stream(stream))
    if st == FS_E_CAPACITY and allow_capacity:
        return int(cnt.value)
    _check(st)
    return int(cnt.value)


def fs_plan(n: int, gens, slices: int, cfg: fs_config | None = None):
    """(order, bounds, leaves): the walk order of the generators, the first
    vector (leaf, 0, 0) of every slice in walk order (rows of -1 past the last
    leaf; the last row is +infinity), and the number of leaves."""
    g, d = _gens(gens)
    order = (ctypes.c_int32 * d)()
    bounds = (ctypes.c_int32 * ((slices + 1) * d))()
    leaves = ctypes.c_uint64(0)
    _check(lib().fs_plan(int(n), g, d, _cfgp_of(cfg), int(slices), order, bounds,
                         ctypes.byref(leaves)))
    rows = [list(bounds[i * d:(i + 1) * d]) for i in range(slices + 1)]
    return list(order), rows, int(leaves.value)


def fs_slice_counts(n: int, gens, slices: int, cfg: fs_config | None = None, stream=None):
    """Per-slice counts of the slicing fs_plan describes."""
    g, d = _gens(gens)
    out = (ctypes.c_uint64 * slices)()
    _check(lib().fs_slice_counts(int(n), g, d, _cfgp_of(cfg), int(slices), out, _stream(stream)))
    return [int(x) for x in out]


def fs_count_noalloc(n: int, gens, dev_count, stream=None) -> None:
    """Enqueue the count using the library's static scratch (no allocation);
    |Z| lands in dev_count[0] (a CUDA 64-bit tensor)."""
    g, d = _gens(gens)
    _check(lib().fs_count_noalloc(int(n), g, d, _ptr(dev_count), _stream(stream)))


def fs_alloc_counts():
    """(device allocations, pinned host allocations) the library has made in
    this process."""
    dv, hv = ctypes.c_uint64(0), ctypes.c_uint64(0)
    lib().fs_alloc_counts(ctypes.byref(dv), ctypes.byref(hv))
    return int(dv.value), int(hv.value)


def _queries(queries):
    arr = (fs_query * len(queries))()
    for i, (n, gens) in enumerate(queries):
        g = [int(x) for x in gens]
        arr[i].n = int(n)
        arr[i].d = len(g)
        for j, x in enumerate(g[:MAX_D]):
            arr[i].gens[j] = x & 0xffffffff
    return arr


def _results(res):
    return [(int(r.count), int(r.min_len), int(r.max_len), int(r.status)) for r in res]


def fs_batch_run(queries, mode: int = BATCH_LENGTHS, cfg: fs_config | None = None, stream=None):
    """[(count, min_len, max_len, status)] for queries = [(n, gens), ...], in one
    persistent launch."""
    q = _queries(queries)
    res = (fs_result * len(queries))()
    _check(lib().fs_batch_run(q, len(queries), int(mode), _cfgp_of(cfg), res, _stream(stream)))
    return _results(res)


def fs_batch_autotune(queries, mode: int = BATCH_LENGTHS, stream=None):
    """(fs_config, ms): the fastest launch shape / work-item count for the batch."""
    q = _queries(queries)
    best = fs_config()
    ms = ctypes.c_double(0)
    _check(lib().fs_batch_autotune(q, len(queries), int(mode), ctypes.byref(best),
                                   ctypes.byref(ms), _stream(stream)))
    return best, float(ms.value)


class Batch:
    """A planned batch of queries: launch() enqueues one evaluation (repeatable,
    capturable in a CUDA graph), results() waits and returns them."""

    def __init__(self, queries, mode: int = BATCH_LENGTHS, cfg: fs_config | None = None):
        self.n = len(queries)
        self._q = _queries(queries)
        h = ctypes.c_void_p(0)
        _check(lib().fs_batch_create(self._q, self.n, int(mode), _cfgp_of(cfg), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib().fs_batch_launch(self._h, _stream(stream)))

    def results(self, stream=None):
        res = (fs_result * self.n)()
        _check(lib().fs_batch_results(self._h, res, _stream(stream)))
        return _results(res)

    def close(self):
        if self._h:
            lib().fs_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fs_reserve(nbytes: int, stream=None) -> None:
    """Grow the scratch of `stream` (default: torch's current stream) to at
    least nbytes now."""
    _check(lib().fs_reserve(int(nbytes), _stream(stream)))


class BatchSlot:
    """A reusable batch for request loops (fs_batch_reserve): load() queries of
    either mode, launch(), then results() after fetch and a wait."""

    def __init__(self, max_queries: int, table_bytes: int, mode: int = BATCH_LENGTHS,
                 cfg: fs_config | None = None):
        h = ctypes.c_void_p(0)
        _check(lib().fs_batch_reserve(int(max_queries), int(table_bytes), int(mode), _cfgp_of(cfg),
                                      ctypes.byref(h)))
        self._h = h
        self.n = 0

    def load(self, queries, mode: int | None = None, stream=None):
        q = _queries(queries)
        if mode is None:
            _check(lib().fs_batch_load(self._h, q, len(queries), _stream(stream)))
        else:
            _check(lib().fs_batch_load_mode(self._h, q, len(queries), int(mode), _stream(stream)))
        self.n = len(queries)

    def launch(self, stream=None):
        _check(lib().fs_batch_launch(self._h, _stream(stream)))
        _check(lib().fs_batch_fetch(self._h, _stream(stream)))

    def results(self):
        import torch
        torch.cuda.synchronize()
        res = (fs_result * self.n)()
        _check(lib().fs_batch_collect(self._h, res))
        return _results(res)

    def close(self):
        if self._h:
            lib().fs_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """The request loop of fs_server_*: submit() queues a request and returns
    its ticket, poll() returns completed responses as dicts.  An ENUMERATE
    response's rows (``rows`` = device address, [count][d] of int16 / int32)
    and a LENGTHS response's histogram (hist=True: floor(n / min g) + 1 uint64
    bins) stay on the device until release(ticket)."""

    def __init__(self, mem_budget_bytes: int = 0, table_bytes: int = 0, max_batch: int = 0,
                 slots: int = 0, window_us: int = 0, job_streams: int = 0,
                 hist_max_leaves: int = 0, direct_leaves: int = 0):
        cfg = fs_server_config(int(mem_budget_bytes), int(table_bytes), int(max_batch),
                               int(slots), int(window_us), int(job_streams), int(hist_max_leaves),
                               int(direct_leaves))
        h = ctypes.c_void_p(0)
        _check(lib().fs_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, op: int, n: int, gens, elem_bytes: int = 2, keep_order: bool = False,
               hist: bool = False) -> int:
        g = [int(x) for x in gens]
        r = fs_request()
        r.n = int(n)
        r.d = len(g)
        for j, x in enumerate(g[:MAX_D]):
            r.gens[j] = x & 0xffffffff
        r.op = int(op)
        r.elem_bytes = int(elem_bytes)
        r.keep_order = 1 if keep_order else 0
        r.hist = 1 if hist else 0
        t = ctypes.c_uint64(0)
        _check(lib().fs_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return int(t.value)

    def poll(self, max_items: int = 256, wait_ms: int = 0):
        out = (fs_response * max_items)()
        got = ctypes.c_int(0)
        _check(lib().fs_server_poll(self._h, out, int(max_items), ctypes.byref(got), int(wait_ms)))
        return [dict(ticket=int(r.ticket), status=int(r.status), op=int(r.op),
                     count=int(r.count), min_len=int(r.min_len), max_len=int(r.max_len),
                     rows=int(r.rows or 0), t_submit=float(r.t_submit),
                     t_start=float(r.t_start), t_counted=float(r.t_counted),
                     t_job=float(r.t_job), t_done=float(r.t_done))
                for r in out[:got.value]]

    def release(self, ticket: int) -> None:
        _check(lib().fs_server_release(self._h, int(ticket)))

    def close(self):
        if self._h:
            lib().fs_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fs_profile_enable(on: bool = True) -> None:
    """Bracket every library kernel launch with CUDA events (for benchmarks)."""
    lib().fs_profile_enable(1 if on else 0)


def fs_profile_only(name: str | None = None) -> None:
    """Record only the kernels timed under `name` (None: every kernel)."""
    lib().fs_profile_only(name.encode() if name else None)


def fs_profile_read(max_entries: int = 64):
    """{kernel name: (launches, total device ms)} recorded since the last read."""
    names = ctypes.create_string_buffer(32 * max_entries)
    launches = (ctypes.c_uint64 * max_entries)()
    ms = (ctypes.c_double * max_entries)()
    k = lib().fs_profile_read(names, launches, ms, max_entries)
    if k < 0:
        raise FsError(FS_E_CUDA, "profile read failed")
    out = {}
    for i in range(k):
        nm = names.raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


def fs_probe_int_rate(kind: int, iters: int = 4096) -> float:
    """GPU-wide 32-bit integer lane-ops/s of kind 0 (add), 1 (lop3), 2 (mad)."""
    out = ctypes.c_double(0)
    _check(lib().fs_probe_int_rate(int(kind), int(iters), ctypes.byref(out)))
    return float(out.value)


def fs_selftest_division(div: int, x0: int, count: int) -> int:
    """Host self test of the invariant-divisor division (no GPU needed)."""
    return int(lib().fs_selftest_division(int(div), int(x0), int(count)))


def fs_selftest_split(leaves: int, slices: int, tail: bool) -> list:
    """The planner's slice starts (host, no GPU): slices + 1 leaf ranks."""
    out = (ctypes.c_uint64 * (int(slices) + 1))()
    _check(lib().fs_selftest_split(int(leaves), int(slices), 1 if tail else 0, out))
    return [int(x) for x in out]
