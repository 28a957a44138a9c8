"""Host-side checks of the C ABI: the library loads, exports every entry
point include/fs.h declares, validates arguments before touching the GPU,
fails loudly without a GPU (no CPU fallback), and its invariant-divisor
division is exact.  None of these launch a kernel."""
import ctypes
import os
import re

import pytest

import paper_2405_07989_gb300 as fs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fs.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(fs_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_loads_and_exports_every_declared_symbol():
    L = fs.lib()
    names = declared_entry_points()
    assert len(names) >= 16
    for name in names:
        assert hasattr(L, name), name
        assert name in fs.SIGNATURES, f"binding lacks {name}"
    assert set(fs.SIGNATURES) == set(names)
    assert fs.fs_version() >= 100


def test_status_strings():
    L = fs.lib()
    for s, name in enumerate(["FS_OK", "FS_E_INVAL", "FS_E_OVERFLOW", "FS_E_CAPACITY",
                              "FS_E_NOMEM", "FS_E_CUDA", "FS_E_TIMEOUT", "FS_E_NOTIMPL"]):
        assert L.fs_status_string(s).decode() == name


def _status(fn, *args):
    try:
        fn(*args)
    except fs.FsError as e:
        return e.status
    return fs.FS_OK


@pytest.mark.parametrize("args,status", [
    ((10, []), fs.FS_E_INVAL),                       # d = 0
    ((10, [3] * 17), fs.FS_E_INVAL),                 # d > 16
    ((10, [3, 0, 5]), fs.FS_E_INVAL),                # zero generator
    ((-1, [3, 5]), fs.FS_E_INVAL),                   # n < 0
    ((2**31 - 5, [3, 5, 7]), fs.FS_E_OVERFLOW),      # n + max g >= 2^31
    ((2**31 - 1, [1]), fs.FS_E_OVERFLOW),
])
def test_argument_validation_before_gpu(args, status):
    assert _status(fs.fs_count, *args) == status


def test_enumerate_argument_validation():
    # elem_bytes, alignment and int16 range are checked before any launch
    st = fs.lib().fs_enumerate(100, (ctypes.c_uint32 * 3)(3, 5, 7), 3, ctypes.c_void_p(16), 10,
                               3, ctypes.byref(ctypes.c_uint64()), None)
    assert st == fs.FS_E_INVAL
    st = fs.lib().fs_enumerate(100, (ctypes.c_uint32 * 3)(3, 5, 7), 3, ctypes.c_void_p(8), 10,
                               4, ctypes.byref(ctypes.c_uint64()), None)
    assert st == fs.FS_E_INVAL  # not 16-byte aligned
    st = fs.lib().fs_enumerate(100000, (ctypes.c_uint32 * 3)(1, 5, 7), 3, ctypes.c_void_p(16),
                               10, 2, ctypes.byref(ctypes.c_uint64()), None)
    assert st == fs.FS_E_OVERFLOW  # int16 cannot hold a coordinate up to 100000
    st = fs.lib().fs_count(10, None, 3, ctypes.byref(ctypes.c_uint64()), None)
    assert st == fs.FS_E_INVAL


def test_count_overflow_bound_refuses_before_gpu():
    """Counts are uint64: a query whose count may reach 2^63 is refused up
    front (the bound (n + sum g)^(d-1) / ((d-1)! prod g)); every workload of
    the benchmarks and tests passes it."""
    import oracle
    from paper_2405_07989_gb300 import workloads
    assert _status(fs.fs_count, 2**30, [1] * 8) == fs.FS_E_OVERFLOW
    assert _status(fs.fs_count, 20000, [5, 6, 7, 8, 9, 10, 11, 12]) == fs.FS_E_OVERFLOW
    assert oracle.count_dp(20000, (5, 6, 7, 8, 9, 10, 11, 12)) > 2**63  # rightly refused
    ok = [workloads.config3(s) for s in range(3)] + [workloads.CONFIG1, workloads.CONFIG2]
    ok += workloads.config4(0) + [(n, g) for _, _, n, g in workloads.config5(0, 2000, 1000.0, 20000)]
    for n, g in ok:
        assert _status(fs.fs_count, n, list(g)) != fs.FS_E_OVERFLOW, (n, g)


def test_cursor_and_host_enumerate_argument_validation():
    L = fs.lib()
    g = (ctypes.c_uint32 * 3)(3, 5, 7)
    h = ctypes.c_void_p(0)
    assert L.fs_cursor_create(100, g, 3, None, 3, None, ctypes.byref(h)) == fs.FS_E_INVAL
    assert L.fs_cursor_create(100000, (ctypes.c_uint32 * 3)(1, 5, 7), 3, None, 2, None,
                              ctypes.byref(h)) == fs.FS_E_OVERFLOW
    assert L.fs_cursor_create(100, g, 3, None, 4, None, None) == fs.FS_E_INVAL
    cnt = ctypes.c_uint64()
    assert L.fs_enumerate_host(100, g, 3, None, None, 10, 4, ctypes.byref(cnt), None) == fs.FS_E_INVAL
    assert L.fs_enumerate_host(100, g, 3, None, None, 0, 5, ctypes.byref(cnt), None) == fs.FS_E_INVAL
    assert L.fs_cursor_next(None, None, 0, ctypes.byref(cnt), None) == fs.FS_E_INVAL
    assert L.fs_cursor_seek(None, 0) == fs.FS_E_INVAL


def test_predicate_validation():
    assert _status(fs.fs_any, 10, [3, 5], [1, 1], 3, 7) == fs.FS_E_INVAL  # op 7
    assert _status(fs.fs_any, 10, [3, 5], [1 << 21, 1], 3, 0) == fs.FS_E_INVAL


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fs.FsError) as e:
        fs.fs_count(500, [5, 7, 11, 13])
    assert e.value.status == fs.FS_E_CUDA
    with pytest.raises(fs.FsError) as e:
        fs.Cursor(500, [5, 7, 11, 13])
    assert e.value.status == fs.FS_E_CUDA
    with pytest.raises(fs.FsError) as e:
        fs.Server()
    assert e.value.status in (fs.FS_E_CUDA, fs.FS_E_NOMEM)


@pytest.mark.parametrize("div", [1, 2, 3, 5, 7, 11, 13, 52, 56, 61, 100, 143, 728, 1000, 4093,
                                 9900, 65535, 65536, 65537, 1 << 20, (1 << 20) + 1,
                                 123456789, 2**30, 2**30 + 1, 2**31 - 1])
def test_invariant_division_exact(div):
    """Granlund-Montgomery division vs C's / and % over ranges of numerators
    around the divisor, its multiples and the top of the 31-bit range."""
    assert fs.fs_selftest_division(div, 0, 1 << 16) == 0
    assert fs.fs_selftest_division(div, 2**31 - (1 << 16), 1 << 16) == 0
    for k in (1, 2, 3, 1000):
        x0 = max(0, min(div * k - 100, 2**31 - 201))
        assert fs.fs_selftest_division(div, x0, 200) == 0


def test_invariant_division_exhaustive_small_divisors():
    for div in range(1, 300):
        assert fs.fs_selftest_division(div, 0, 20000) == 0


@pytest.mark.parametrize("leaves,slices", [(0, 1), (1, 1), (5, 16), (1000, 16), (1000, 17),
                                           (10**6, 38912), (3832670754382, 155648),
                                           (16614104, 38912), (100, 1000), (2**62, 3)])
def test_slice_split_covers_and_balances(leaves, slices):
    """The planner's split: slice starts from 0 to the leaf count, never
    decreasing.  Equal split: sizes differ by at most one.  With the tail (the
    planner's own slice count): the first slices equal to within one, the last
    sixteenth equal to within one and about a sixteenth of the others."""
    for tail in (False, True):
        st = fs.fs_selftest_split(leaves, slices, tail)
        assert len(st) == slices + 1 and st[0] == 0 and st[-1] == leaves
        sizes = [b - a for a, b in zip(st, st[1:])]
        assert min(sizes) >= 0
        nt = slices // 16 if tail else 0
        head, tl = sizes[:slices - nt], sizes[slices - nt:]
        assert max(head) - min(head) <= 1, (tail, leaves, slices)
        if not tail or nt == 0:
            assert max(sizes) - min(sizes) <= 1
            assert st == [s * (leaves // slices) + min(s, leaves % slices) for s in range(slices + 1)]
            continue
        assert max(tl) - min(tl) <= 1
        if min(head) >= 64:  # the tail slices are a sixteenth of a head slice (rounding aside)
            ratio = (sum(tl) / len(tl)) / (sum(head) / len(head))
            assert abs(ratio - 1 / 16) < 1e-3 + 2 / min(head), ratio
    with pytest.raises(fs.FsError):
        fs.fs_selftest_split(10, 0, True)
