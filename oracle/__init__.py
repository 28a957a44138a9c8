"""CPU oracle for factorization sets (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does: it has
no CPU fallback, and it shares no code with this oracle.

The arithmetic lives in ``oracle.c`` (plain single-threaded C); this module
compiles it on first use with gcc and wraps it with ctypes.  Functions and the
paper passages they follow:

* :func:`enumerate_stream` / :func:`enumerate_range` -- the bounded lexicographic
  stream: first candidate (Sec. 3.2.1) and Algorithm 3.1, filtered by wasValid.
* :func:`range_stats` -- count / min / max / histogram consumers on that stream
  (Sec. 2).
* :func:`any_pred` -- predicate consumer on that stream (Sec. 2).
* :func:`brute` -- the definition of Z(n, g) (Sec. 1) over the box of Thm 3.3.
* :func:`count_dp`, :func:`length_dp`, :func:`minmax_dp` -- plain definitions of
  the count and the length statistics as generating-function coefficients.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no architecture flags)."""
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_enumerate_range.restype = ctypes.c_int64
            lib.oracle_enumerate_range.argtypes = [
                ctypes.c_int64, _u32p, ctypes.c_int, _i64p, _i64p, _i32p, ctypes.c_int64, _u64p]
            lib.oracle_range_stats.restype = ctypes.c_int
            lib.oracle_range_stats.argtypes = [
                ctypes.c_int64, _u32p, ctypes.c_int, _i64p, _i64p, _u64p, _i64p, _i64p,
                _u64p, ctypes.c_int64, _u64p]
            lib.oracle_any.restype = ctypes.c_int
            lib.oracle_any.argtypes = [ctypes.c_int64, _u32p, ctypes.c_int, _i32p,
                                       ctypes.c_int64, ctypes.c_int, ctypes.c_uint32]
            lib.oracle_brute.restype = ctypes.c_int64
            lib.oracle_brute.argtypes = [ctypes.c_int64, _u32p, ctypes.c_int, _i32p,
                                         ctypes.c_int64]
            lib.oracle_count_dp.restype = ctypes.c_int
            lib.oracle_count_dp.argtypes = [ctypes.c_int64, _u32p, ctypes.c_int, _u64p]
            lib.oracle_length_dp.restype = ctypes.c_int
            lib.oracle_length_dp.argtypes = [ctypes.c_int64, _u32p, ctypes.c_int, _u64p,
                                             ctypes.c_int64]
            lib.oracle_minmax_dp.restype = ctypes.c_int
            lib.oracle_minmax_dp.argtypes = [ctypes.c_int64, _u32p, ctypes.c_int, _i64p, _i64p]
            lib.oracle_set_mutation.restype = None
            lib.oracle_set_mutation.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _gens(gens) -> np.ndarray:
    g = np.ascontiguousarray(np.asarray(gens, dtype=np.uint32))
    if g.ndim != 1 or g.size < 1 or np.any(g == 0):
        raise ValueError("generators must be a nonempty list of positive integers")
    return g


def _vec(v, d):
    if v is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int64))
    if a.shape != (d,):
        raise ValueError("bound must have d coordinates")
    return a, a.ctypes.data_as(_i64p)


def set_mutation(k: int) -> None:
    """Switch on one deliberately wrong variant of the oracle (0 = faithful).

    Used only by the pin tests, to show that each pin catches a plausible
    mistake in the oracle."""
    _load().oracle_set_mutation(int(k))


def hist_len(n: int, gens) -> int:
    """Number of length bins: lengths run over 0..floor(n / min g)."""
    return int(n) // int(min(int(x) for x in gens)) + 1


def enumerate_range(n: int, gens, lo=None, hi=None, cap: int | None = None):
    """Factorizations in the lex slice [lo, hi) in the paper's (decreasing) order.

    Returns (rows int32 [count, d], candidates).  lo=None is (0,..,0); hi=None
    is +infinity.  cap limits the rows stored (the count is always exact)."""
    lib = _load()
    g = _gens(gens)
    d = g.size
    lo_a, lo_p = _vec(lo, d)
    hi_a, hi_p = _vec(hi, d)
    cand = ctypes.c_uint64(0)
    if cap is None:
        cnt = lib.oracle_enumerate_range(int(n), g.ctypes.data_as(_u32p), d, lo_p, hi_p,
                                         None, 0, ctypes.byref(cand))
        cap = cnt
    out = np.zeros((max(cap, 1), d), dtype=np.int32)
    cnt = lib.oracle_enumerate_range(int(n), g.ctypes.data_as(_u32p), d, lo_p, hi_p,
                                     out.ctypes.data_as(_i32p), int(cap), ctypes.byref(cand))
    return out[:min(cnt, cap)], int(cand.value)


def enumerate_stream(n: int, gens):
    """The whole stream of Algorithm 3.1 (lex-decreasing) and its candidate count."""
    return enumerate_range(n, gens, None, None)


def enumerate_sorted(n: int, gens) -> np.ndarray:
    """Z(n, g) as int32 rows in lex-ASCENDING order (the stream, reversed)."""
    rows, _ = enumerate_stream(n, gens)
    return rows[::-1].copy()


def range_stats(n: int, gens, lo=None, hi=None, with_hist: bool = True):
    """(count, min_len, max_len, hist or None, candidates) over the slice [lo, hi)."""
    lib = _load()
    g = _gens(gens)
    d = g.size
    lo_a, lo_p = _vec(lo, d)
    hi_a, hi_p = _vec(hi, d)
    hl = hist_len(n, g)
    hist = np.zeros(hl, dtype=np.uint64) if with_hist else None
    cnt = ctypes.c_uint64(0)
    mn = ctypes.c_int64(0)
    mx = ctypes.c_int64(0)
    cand = ctypes.c_uint64(0)
    rc = lib.oracle_range_stats(int(n), g.ctypes.data_as(_u32p), d, lo_p, hi_p,
                                ctypes.byref(cnt), ctypes.byref(mn), ctypes.byref(mx),
                                hist.ctypes.data_as(_u64p) if with_hist else None,
                                hl if with_hist else 0, ctypes.byref(cand))
    if rc != 0:
        raise RuntimeError("length outside the histogram range")
    return int(cnt.value), int(mn.value), int(mx.value), hist, int(cand.value)


def any_pred(n: int, gens, w, c: int, op: int = 0, modulus: int = 0) -> bool:
    """True iff some factorization a has sum w_i a_i (op) c, or == c mod modulus."""
    lib = _load()
    g = _gens(gens)
    wa = np.zeros(g.size, dtype=np.int32)
    wa[:len(w)] = np.asarray(w, dtype=np.int64)[:g.size]
    return bool(lib.oracle_any(int(n), g.ctypes.data_as(_u32p), g.size,
                               wa.ctypes.data_as(_i32p), int(c), int(op), int(modulus)))


def brute(n: int, gens) -> np.ndarray:
    """Z(n, g) by brute force over the box a_i <= n / g_i, lex-ascending."""
    lib = _load()
    g = _gens(gens)
    cnt = lib.oracle_brute(int(n), g.ctypes.data_as(_u32p), g.size, None, 0)
    out = np.zeros((max(cnt, 1), g.size), dtype=np.int32)
    lib.oracle_brute(int(n), g.ctypes.data_as(_u32p), g.size, out.ctypes.data_as(_i32p), cnt)
    return out[:cnt]


def count_dp(n: int, gens) -> int:
    """|Z(n, g)| as [x^n] prod 1/(1 - x^{g_i}) (exact; raises on 64-bit overflow)."""
    lib = _load()
    g = _gens(gens)
    out = ctypes.c_uint64(0)
    rc = lib.oracle_count_dp(int(n), g.ctypes.data_as(_u32p), g.size, ctypes.byref(out))
    if rc != 0:
        raise OverflowError("count does not fit 64 bits" if rc == -1 else "out of memory")
    return int(out.value)


def length_dp(n: int, gens) -> np.ndarray:
    """Histogram of sum a_i over Z(n, g) as [x^n y^l] prod 1/(1 - y x^{g_i})."""
    lib = _load()
    g = _gens(gens)
    hl = hist_len(n, g)
    hist = np.zeros(hl, dtype=np.uint64)
    rc = lib.oracle_length_dp(int(n), g.ctypes.data_as(_u32p), g.size,
                              hist.ctypes.data_as(_u64p), hl)
    if rc != 0:
        raise OverflowError("histogram overflow" if rc == -1 else "out of memory")
    return hist


def minmax_dp(n: int, gens):
    """(min, max) of sum a_i over Z(n, g), or None if Z is empty."""
    lib = _load()
    g = _gens(gens)
    mn = ctypes.c_int64(0)
    mx = ctypes.c_int64(0)
    ok = lib.oracle_minmax_dp(int(n), g.ctypes.data_as(_u32p), g.size, ctypes.byref(mn),
                              ctypes.byref(mx))
    if ok < 0:
        raise MemoryError("out of memory")
    return (int(mn.value), int(mx.value)) if ok else None


def pred_holds_rows(rows: np.ndarray, w, c: int, op: int = 0, modulus: int = 0) -> np.ndarray:
    """Evaluate the linear predicate on explicit rows (tests on tiny inputs)."""
    rows = np.asarray(rows, dtype=np.int64)
    wa = np.zeros(rows.shape[1], dtype=np.int64)
    wa[:len(w)] = np.asarray(w, dtype=np.int64)[:rows.shape[1]]
    s = rows @ wa
    if modulus > 0:
        return np.mod(s, modulus) == (int(c) % int(modulus))
    if op == 0:
        return s == c
    if op == 1:
        return s <= c
    return s >= c
