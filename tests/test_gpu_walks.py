"""The two ways the order-free walks take a group of sibling runs give the same
exact results (through the C ABI, against the CPU oracle).

fs_config.walk forces one way for every group: PACKED (each run's full 32-leaf
steps, then the runs' remainders packed into shared steps) or LANES (lane j
walks sibling run j alone); AUTO picks per group.  Each consumer that walks in
either way -- count (PAIR and the trailing-table walks), length statistics and
histogram, the predicate, per-slice counts, the batched walk -- is checked
under all three against the oracle's DPs, its bounded streams and brute force.
"""
import numpy as np
import pytest

import oracle
import paper_2405_07989_gb300 as fs
from paper_2405_07989_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WALKS = {"auto": fs.WALK_AUTO, "packed": fs.WALK_PACKED, "lanes": fs.WALK_LANES}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fs.lib()
    yield
    torch.cuda.synchronize()


def cases():
    out = workloads.random_medium(seed=33, count=40, d_lo=3, d_hi=9, g_lo=2, g_hi=40,
                                  n_lo=0, n_hi=400)
    # long runs (innermost generator small against n), few siblings, common divisors
    out += [(3000, (11, 13, 17, 19, 23, 29)), (2500, (5, 7, 11, 13)), (1500, (3, 5, 97)),
            (2000, (61, 3, 4)), (4000, (172, 61, 52, 124, 95, 89, 56, 142)),
            (401, (4, 6, 8, 10)), (420, (30, 42, 70, 105, 11)), (900, (35, 21, 15, 9, 25, 49)),
            (1000, (100, 60, 36, 24, 18, 8, 12)), (513, (2, 4, 6, 8, 10)), (97, (1, 1, 1)),
            (0, (3, 5, 7)), (500, (7, 7, 7, 7)), workloads.CONFIG1]
    return out


def cfg(walk, method=fs.METHOD_PAIR, keep_order=False, slices=0):
    return fs.make_config(method=method, keep_order=keep_order, slices=slices, walk=walk)


def test_walk_mode_is_validated():
    with pytest.raises(fs.FsError) as e:
        fs.fs_count(100, (3, 5, 7), fs.make_config(walk=3))
    assert e.value.status == fs.FS_E_INVAL


@pytest.mark.parametrize("walk", list(WALKS))
def test_count_every_method(walk):
    w = WALKS[walk]
    for n, g in cases():
        expect = oracle.count_dp(n, g)
        assert fs.fs_count(n, g, cfg(w)) == expect, (n, g)
        assert fs.fs_count(n, g, cfg(w, keep_order=True)) == expect, (n, g)
        if len(g) >= 4:
            assert fs.fs_count(n, g, cfg(w, fs.METHOD_TRIPLE)) == expect, (n, g)
        if len(g) >= 5:
            assert fs.fs_count(n, g, cfg(w, fs.METHOD_QUAD)) == expect, (n, g)


@pytest.mark.parametrize("walk", list(WALKS))
def test_lengths_and_histogram(walk):
    w = WALKS[walk]
    for n, g in cases():
        hl = oracle.hist_len(n, g)
        ref = oracle.length_dp(n, g)
        mm = oracle.minmax_dp(n, g) or (0, 0)
        for keep in (False, True):
            hist = torch.full((hl + 2,), 777, dtype=torch.int64, device="cuda")
            got = fs.fs_length_stats(n, g, hist, cfg(w, keep_order=keep))
            assert got == (int(ref.sum()),) + tuple(mm), (n, g, keep)
            h = hist.cpu().numpy()
            assert np.array_equal(h[:hl].astype(np.uint64), ref), (n, g, keep)
            assert np.all(h[hl:] == 777)
        if len(g) >= 4:
            assert fs.fs_length_stats(n, g, None, cfg(w, fs.METHOD_TRIPLE)) == \
                (int(ref.sum()),) + tuple(mm), (n, g)


@pytest.mark.parametrize("walk", list(WALKS))
def test_any(walk):
    w = WALKS[walk]
    rng = np.random.default_rng(5)
    for n, g in cases():
        if n > 1000:
            continue
        rows = oracle.enumerate_sorted(n, g)
        d = len(g)
        for _ in range(4):
            wt = [int(x) for x in rng.integers(-3, 4, size=d)]
            op = int(rng.integers(0, 3))
            modulus = int(rng.choice([0, 0, 3, 7]))
            if rows.shape[0] and rng.random() < 0.6:
                r = rows[int(rng.integers(0, rows.shape[0]))].astype(np.int64)
                c = int(np.dot(r, np.asarray(wt, dtype=np.int64))) + int(rng.integers(-1, 2))
            else:
                c = int(rng.integers(-20, 80))
            expect = bool(oracle.pred_holds_rows(rows, wt, c, op, modulus).any()) \
                if rows.shape[0] else False
            assert fs.fs_any(n, g, wt, c, op, modulus, cfg(w)) == expect, (n, g, wt, c, op)


@pytest.mark.parametrize("walk", ["packed", "lanes"])
@pytest.mark.parametrize("method", [fs.METHOD_PAIR, fs.METHOD_TRIPLE], ids=["pair", "triple"])
def test_slice_counts_match_oracle_streams(walk, method):
    """Slices cut runs anywhere: the first and last run of a slice are partial."""
    w = WALKS[walk]
    for n, g in [(1500, (29, 23, 19, 17, 13, 11)), (2000, (61, 52, 56, 89)),
                 (401, (4, 6, 8, 10)), (900, (35, 21, 15, 9, 25, 49))]:
        for slices in (1, 7, 300):
            c = cfg(w, method)
            order, bounds, leaves = fs.fs_plan(n, g, slices, c)
            counts = fs.fs_slice_counts(n, g, slices, c)
            assert sum(counts) == oracle.count_dp(n, g)
            wg = [g[i] for i in order]
            rng = np.random.default_rng(slices)
            for s in rng.choice(slices, min(slices, 12), replace=False):
                lo = bounds[s]
                if lo[0] < 0:
                    assert counts[s] == 0
                    continue
                hi = bounds[s + 1] if bounds[s + 1][0] >= 0 else None
                ref, _, _, _, _ = oracle.range_stats(n, wg, lo, hi, with_hist=False)
                assert counts[s] == ref, (n, g, slices, s)


@pytest.mark.parametrize("walk", list(WALKS))
def test_batch(walk):
    w = WALKS[walk]
    qs = workloads.config4(0, nq=256)
    qs += [(n, g) for n, g in cases() if len(g) >= 3]
    for mode in (fs.BATCH_COUNT, fs.BATCH_LENGTHS):
        for method in (fs.METHOD_PAIR, fs.METHOD_AUTO):
            with fs.Batch(qs, mode, fs.make_config(method=method, walk=w)) as b:
                b.launch()
                res = b.results()
            for (n, g), r in zip(qs, res):
                assert r[0] == oracle.count_dp(n, g), (n, g)
                if mode == fs.BATCH_LENGTHS and r[0] > 0:
                    assert tuple(r[1:3]) == oracle.minmax_dp(n, g), (n, g)


@pytest.mark.parametrize("walk", ["packed", "lanes"])
def test_config3_count_forced(walk):
    """The heavy count-only query at full size through the PAIR walk."""
    n, g = workloads.config3(0)
    assert fs.fs_count(n, g, cfg(WALKS[walk])) == 7655692813487


@pytest.mark.parametrize("walk", list(WALKS))
def test_trailing_walks_sibling_stride_even(walk):
    """Trailing-table walks whose sibling runs have residuals an even distance
    apart (2, 4, .., 32 and more times an odd number) and an odd step inside a
    run: the walk holds lanes back to spread their table reads over the banks.
    Counts, per-slice counts and the length range against the oracle's DPs."""
    w = WALKS[walk]
    cases = []
    for sib in (2 * 31, 4 * 15, 8 * 7, 16 * 5, 32 * 3, 64):
        # generators in descending (walk) order; the walked levels end with the
        # sibling level `sib` and an odd run level
        cases.append((2500, (sib + 41, sib + 17, sib, 45, 31, 29, 23, 19)))  # QUAD walks 4 levels
        cases.append((2500, (sib + 41, sib, 45, 29, 23, 19)))                # TRIPLE walks 3
        cases.append((900, (sib + 3, sib, 33, 25, 9, 7, 5)))                 # QUAD walks 3
    for n, g in cases:
        expect = oracle.count_dp(n, g)
        for method in (fs.METHOD_TRIPLE, fs.METHOD_QUAD, fs.METHOD_AUTO):
            if method == fs.METHOD_QUAD and len(g) < 5:
                continue
            c = cfg(w, method)
            assert fs.fs_count(n, g, c) == expect, (n, g, method)
            counts = fs.fs_slice_counts(n, g, 37, c)
            assert sum(counts) == expect, (n, g, method)
        mm = oracle.minmax_dp(n, g) or (0, 0)
        assert fs.fs_length_stats(n, g, None, cfg(w, fs.METHOD_TRIPLE)) == (expect,) + tuple(mm)


@pytest.mark.parametrize("n", [262160, 262161])
def test_pair_count_quotient_by_lcm_near_the_multiply_high_limit(n):
    """The PAIR count walk takes floor(r / lcm) as one multiply-high while
    n lcm < 2^32 and by the general division above it: lcm(127, 129) = 16383,
    so n = 262160 is the last inside and n = 262161 the first outside."""
    for g in ((100003, 127, 129, 131), (100003, 127, 129)):
        expect = oracle.count_dp(n, g)
        assert fs.fs_count(n, g, cfg(fs.WALK_AUTO)) == expect, (n, g)
        assert fs.fs_count(n, g, cfg(fs.WALK_LANES)) == expect, (n, g)


def brute_hist(n, g):
    """Histogram of sum a_i over Z(n, g) for g = (huge, c, a, b) with huge > n:
    every factorization has a_0 = 0; the rest by direct summation."""
    big, c, a, b = g
    assert big > n
    h = np.zeros(n // min(g) + 1, dtype=np.uint64)
    for k in range(n // c + 1):
        r = n - k * c
        x = np.arange(r // a + 1, dtype=np.int64)
        y, rem = np.divmod(r - a * x, b)
        ok = rem == 0
        np.add.at(h, k + x[ok] + y[ok], 1)
    return h


@pytest.mark.parametrize("n", [1398101, 1398112])
def test_pair_histogram_quotient_by_lcm_near_the_multiply_high_limit(n):
    """The same for the histogram walk with per-warp difference arrays (pair
    tables up to lcm 4096, the arrays of a block within 64 KB): lcm(1536,
    3072) = 3072, n = 1398101 the last inside, n = 1398112 outside; every
    bin against direct summation."""
    g = (2000003, 3083, 3072, 1536)
    ref = brute_hist(n, g)
    hist = torch.zeros(ref.size, dtype=torch.int64, device="cuda")
    got = fs.fs_length_stats(n, g, hist, cfg(fs.WALK_AUTO))
    assert got[0] == int(ref.sum()) == oracle.count_dp(n, g)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), ref), n


@pytest.mark.parametrize("walk", ["auto", "lanes"])
def test_trailing_length_range_both_paths(walk):
    """The length range from the trailing tables: two walks with the tables in
    shared memory (the count, then minimum and maximum packed in 16 bits) while
    the table fits 160 KB, one walk through L2 above (n >= 40960).  Count,
    minimum and maximum against the oracle's DPs, both sides of that size."""
    w = WALKS[walk]
    for n in (3000, 40959, 40960, 45000):
        for g in ((97, 89, 83, 79, 73), (64, 61, 59, 53, 47, 43), (124, 95, 89, 61, 56, 52)):
            expect = (oracle.count_dp(n, g),) + tuple(oracle.minmax_dp(n, g) or (0, 0))
            for method in (fs.METHOD_TRIPLE, fs.METHOD_QUAD, fs.METHOD_AUTO):
                assert fs.fs_length_stats(n, g, None, cfg(w, method)) == expect, (n, g, method)


def brute_count_minmax3(n, g):
    """|Z(n, g)| and its length range for three generators by direct
    summation: every (a, x) with the third coordinate solved (numpy)."""
    g0, g1, g2 = g
    c, lo, hi = 0, None, None
    x = np.arange(n // g1 + 1, dtype=np.int64)
    for a in range(n // g0 + 1):
        rest = n - a * g0 - x * g1
        ok = (rest >= 0) & (rest % g2 == 0)
        if ok.any():
            tot = a + x[ok] + rest[ok] // g2
            c += int(ok.sum())
            lo = int(tot.min()) if lo is None else min(lo, int(tot.min()))
            hi = int(tot.max()) if hi is None else max(hi, int(tot.max()))
    return c, (lo, hi) if c else (0, 0)


@pytest.mark.parametrize("g", [(99991, 70001, 50021), (99991, 70001, 46337)])
def test_pair_first_solution_both_remainder_paths(g):
    """Without pair tables (lcm above the table limit) a leaf's first solution
    is t u^-1 mod v: one invariant division while v^2 < 2^31 (v = 46337
    here), a 64-bit remainder above (v = 50021).  Count and length range of
    the PAIR walk at n = 2e9 against direct summation."""
    n = 2_000_000_011
    c, mm = brute_count_minmax3(n, g)
    assert c > 1000
    assert fs.fs_count(n, g, cfg(fs.WALK_AUTO)) == c, g
    assert fs.fs_length_stats(n, g, None, cfg(fs.WALK_AUTO)) == (c,) + mm, g
