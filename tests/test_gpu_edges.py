"""Edge cases through the C ABI against the oracle: the largest dimension
(d = 16, the generic write walk), repeated generators at d = 16, one and two
generators, an element near the 2^31 limit, the int16 boundary, empty sets,
and every method on the same inputs."""
import numpy as np
import pytest

import oracle
import paper_2405_07989_gb300 as fs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fs.lib()


def rows_sorted(n, g, elem_bytes=4, cfg=None):
    c = fs.fs_count(n, g)
    dt = torch.int16 if elem_bytes == 2 else torch.int32
    out = torch.empty((max(c, 1), len(g)), dtype=dt, device="cuda")
    assert fs.fs_enumerate(n, g, out, cap=c, elem_bytes=elem_bytes, cfg=cfg) == c
    a = out[:c].cpu().numpy().astype(np.int64)
    return a[np.lexsort(a.T[::-1])] if c else a


def check_all(n, g):
    c = oracle.count_dp(n, g)
    for m in (fs.METHOD_AUTO, fs.METHOD_PAIR, fs.METHOD_PLAIN):
        assert fs.fs_count(n, g, fs.make_config(method=m)) == c, (n, g, m)
    mm = oracle.minmax_dp(n, g) or (0, 0)
    hist = torch.zeros(oracle.hist_len(n, g), dtype=torch.int64, device="cuda")
    assert fs.fs_length_stats(n, g, hist) == (c,) + tuple(mm)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), oracle.length_dp(n, g))
    ref = oracle.enumerate_sorted(n, g).astype(np.int64).reshape(-1, len(g))
    assert np.array_equal(rows_sorted(n, g), ref)
    w = list(range(1, len(g) + 1))
    target = int((ref @ np.array(w)).max()) if c else 0
    assert fs.fs_any(n, g, w, target) == (c > 0)
    assert not fs.fs_any(n, g, w, target + 1, op=2)  # nothing exceeds the maximum


def test_sixteen_generators():
    rng = np.random.default_rng(7)
    g = tuple(int(x) for x in rng.choice(np.arange(40, 201), 16, replace=False))
    for n in (0, 39, 250, 420):
        check_all(n, g)


def test_sixteen_equal_generators():
    """d = 16 copies of 7: |Z(7m)| = C(m + 15, 15) distinct rows."""
    g = (7,) * 16
    for n in (0, 6, 7, 35, 49):
        check_all(n, g)
    assert fs.fs_count(70, g) == 3268760  # C(25, 15)


def test_one_and_two_generators():
    for n, g in [(0, (5,)), (35, (5,)), (36, (5,)), (2**31 - 8, (7,)), (2**31 - 9, (7,)),
                 (1000, (6, 10)), (999, (6, 10)), (12345, (97, 101)), (1, (1, 1))]:
        c = oracle.count_dp(n, g) if n < 10**6 else int(n % g[0] == 0)
        assert fs.fs_count(n, g) == c, (n, g)
        if n < 10**6:
            check_all(n, g)


def test_element_near_the_limit():
    """n + max g just below 2^31 with large generators (few factorizations):
    counted and listed; one more and the query is refused."""
    g = (1000000007, 700000001, 500000003)
    n = 2**31 - 1 - max(g)
    rows, _ = oracle.enumerate_stream(n, g)
    c = rows.shape[0]
    assert fs.fs_count(n, g) == c
    out = torch.empty((max(c, 1), 3), dtype=torch.int32, device="cuda")
    assert fs.fs_enumerate(n, g, out, cap=c) == c
    mine = out[:c].cpu().numpy().astype(np.int64)
    assert sorted(map(tuple, mine)) == sorted(map(tuple, rows.astype(np.int64)))
    with pytest.raises(fs.FsError) as e:
        fs.fs_count(n + 1, g)
    assert e.value.status == fs.FS_E_OVERFLOW


def test_int16_boundary():
    """int16 rows hold coordinates up to 32767: n / min g = 32767 is allowed,
    32768 is refused."""
    g = (1, 40000, 50000)
    n = 32767
    c = oracle.count_dp(n, g)
    assert np.array_equal(rows_sorted(n, g, elem_bytes=2),
                          oracle.enumerate_sorted(n, g).astype(np.int64).reshape(-1, 3))
    with pytest.raises(fs.FsError) as e:
        out = torch.empty((4, 3), dtype=torch.int16, device="cuda")
        fs.fs_enumerate(32768, g, out, cap=4, elem_bytes=2)
    assert e.value.status == fs.FS_E_OVERFLOW
    assert c > 0


def test_empty_sets_every_method():
    for n, g in [(1, (2, 3)), (11, (4, 6, 8, 10)), (7, (8, 9, 10, 11, 12))]:
        for m in (fs.METHOD_AUTO, fs.METHOD_PAIR, fs.METHOD_PLAIN):
            cfg = fs.make_config(method=m)
            assert fs.fs_count(n, g, cfg) == 0
            out = torch.full((4, len(g)), -5, dtype=torch.int32, device="cuda")
            assert fs.fs_enumerate(n, g, out, cap=4, cfg=cfg) == 0
            assert bool((out == -5).all())
            assert fs.fs_length_stats(n, g, None, cfg) == (0, 0, 0)


def _lattice_reference(n, g):
    """For g = (H, 1, A, B): |Z| and the length range by direct summation over
    a_0 and x (a_1 takes up whatever x A + y B leaves of n - a_0 H)."""
    H, _, A, B = g
    total, lo, hi = 0, None, None
    for a0 in range(n // H + 1):
        R = n - a0 * H
        for x in range(R // A + 1):
            ymax = (R - x * A) // B
            total += ymax + 1
            shortest = a0 + (R - x * A - ymax * B) + x + ymax  # a_1 smallest
            lo = shortest if lo is None else min(lo, shortest)
        hi = max(hi or 0, a0 + R)  # x = y = 0: a_1 = R
    return total, lo, hi


def test_sibling_runs_with_more_than_two_to_the_31_leaves():
    """Runs of up to 10^9 leaves each (generator 1 innermost, 8 sibling runs):
    the walks take a sibling group's runs only while their leaves stay below
    2^31 and continue with the next group.  The pair (200000, 300000) has
    common divisor 10^5, so the length walk (which skips) visits one leaf in
    10^5 and can take the whole set as a single slice, which crosses that cap
    twice.  Count and length range against a direct summation; the
    ordered rows are valid factorizations, strictly lex-ascending, and as many
    as the count: that is Z, in order.  (The leaf-count table of this query
    takes 7.5 GiB, under the library's 8 GiB limit.)"""
    g = (1 << 27, 1, 200000, 300000)
    n = 10**9
    Z, lo, hi = _lattice_reference(n, g)
    assert (Z, lo, hi) == (25066630, 3334, 10**9)
    for keep in (True, False):
        assert fs.fs_count(n, g, fs.make_config(keep_order=keep)) == Z, keep
    for keep, slices in ((True, 0), (True, 1), (False, 0)):
        cfg = fs.make_config(keep_order=keep, slices=slices)
        assert fs.fs_length_stats(n, g, None, cfg) == (Z, lo, hi), (keep, slices)
    out = torch.full((Z, 4), -1, dtype=torch.int32, device="cuda")
    gt = torch.tensor(g, dtype=torch.int64, device="cuda")
    assert fs.fs_enumerate(n, g, out, cap=Z, cfg=fs.make_config(keep_order=True)) == Z
    assert bool(((out.long() * gt).sum(1) == n).all())
    diff = out[1:].long() - out[:-1].long()
    nz = diff != 0
    first = nz.to(torch.int32).argmax(1, keepdim=True)
    assert bool(nz.any(1).all()) and bool((diff.gather(1, first) > 0).all())
    del out, diff, nz, first
    torch.cuda.empty_cache()
