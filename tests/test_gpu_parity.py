"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything here is exact integer arithmetic, so the bar is bit-exactness:
counts, min / max lengths and histograms equal the oracle's; enumerated rows,
sorted, equal the oracle's set row for row, and the GPU's own order is
checked to be lex-ascending in the walk order.
"""
import numpy as np
import pytest

import oracle
import paper_2405_07989_gb300 as fs
from paper_2405_07989_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fs.lib()
    yield
    torch.cuda.synchronize()


PLAIN = fs.make_config(method=fs.METHOD_PLAIN)
PAIR = fs.make_config(method=fs.METHOD_PAIR)
PLAIN_KEEP = fs.make_config(method=fs.METHOD_PLAIN, keep_order=True)
PAIR_KEEP = fs.make_config(method=fs.METHOD_PAIR, keep_order=True)
CONFIGS = {"pair": PAIR, "plain": PLAIN, "pair_keep": PAIR_KEEP, "plain_keep": PLAIN_KEEP}
TRIPLE = fs.make_config(method=fs.METHOD_TRIPLE)
TRIPLE_KEEP = fs.make_config(method=fs.METHOD_TRIPLE, keep_order=True)
QUAD = fs.make_config(method=fs.METHOD_QUAD)
QUAD_KEEP = fs.make_config(method=fs.METHOD_QUAD, keep_order=True)
AUTO = fs.make_config()


def lexsort_rows(a):
    a = np.asarray(a)
    if a.shape[0] == 0:
        return a
    idx = np.lexsort(a.T[::-1])
    return a[idx]


def gpu_enumerate(n, gens, cfg=None, elem_bytes=4, cap=None, extra_rows=0):
    d = len(gens)
    cnt = fs.fs_count(n, gens, cfg)
    rows = cnt + extra_rows if cap is None else cap
    dtype = torch.int32 if elem_bytes == 4 else torch.int16
    out = torch.full((max(rows, 1) * d + 8,), -7, dtype=dtype, device="cuda")
    got = fs.fs_enumerate(n, gens, out, cap=rows, elem_bytes=elem_bytes, cfg=cfg,
                          allow_capacity=True)
    torch.cuda.synchronize()
    return got, out


def medium_cases():
    cases = workloads.random_medium(seed=21, count=60, d_lo=1, d_hi=9, g_lo=2, g_hi=40,
                                    n_lo=0, n_hi=350)
    cases += [(0, (3, 5, 7)), (0, (2,)), (17, (5,)), (20, (5,)), (10, (5, 5)),
              (40, (40, 1)), (97, (1, 1, 1)), (300, (1, 2, 3, 4)), (60, (61, 7, 5)),
              (500, (7, 7, 7, 7)), (250, (6, 10, 15)), (123, (4, 6, 8, 10)),
              workloads.CONFIG1]
    return cases


# ---------------------------------------------------------------------------
# count
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("method", list(CONFIGS))
def test_count_random(method):
    cfg = CONFIGS[method]
    for n, g in medium_cases():
        assert fs.fs_count(n, g, cfg) == oracle.count_dp(n, g), (n, g)


@pytest.mark.parametrize("cfg", [TRIPLE, TRIPLE_KEEP, QUAD, QUAD_KEEP, AUTO],
                         ids=["triple", "triple_keep", "quad", "quad_keep", "auto"])
def test_count_triple(cfg):
    """The trailing-three and trailing-four tables (Sec. 6.1) give the same
    counts; explicit TRIPLE refuses d < 4, QUAD d < 5, AUTO falls back to the
    shallower tables or PAIR there."""
    dmin = 5 if cfg in (QUAD, QUAD_KEEP) else 4
    for n, g in medium_cases():
        if len(g) < dmin and cfg is not AUTO:
            with pytest.raises(fs.FsError) as e:
                fs.fs_count(n, g, cfg)
            assert e.value.status == fs.FS_E_NOTIMPL
            continue
        assert fs.fs_count(n, g, cfg) == oracle.count_dp(n, g), (n, g)


def test_length_min_max_triple():
    """fs_length_stats without a histogram (TRIPLE under AUTO): count, min, max."""
    for n, g in medium_cases():
        mm = oracle.minmax_dp(n, g) or (0, 0)
        expect = (oracle.count_dp(n, g),) + tuple(mm)
        assert fs.fs_length_stats(n, g, None, AUTO) == expect, (n, g)
        if len(g) >= 4:
            assert fs.fs_length_stats(n, g, None, TRIPLE) == expect, (n, g)
        if len(g) >= 5:
            assert fs.fs_length_stats(n, g, None, QUAD) == expect, (n, g)
    with pytest.raises(fs.FsError) as e:  # a histogram needs the PAIR walk
        h = torch.zeros(1000, dtype=torch.int64, device="cuda")
        fs.fs_length_stats(300, (11, 13, 17, 19), h, TRIPLE)
    assert e.value.status == fs.FS_E_NOTIMPL


def test_count_table1_pins_and_errata():
    """Table 1's cells: the GPU reproduces the exact count (the printed value
    for the 26 pinned cells, the oracle's for the three errata)."""
    import test_oracle as t
    for gens, n, printed, status in t.table1_cells():
        got = fs.fs_count(n, gens)
        assert got == oracle.count_dp(n, gens)
        if status == "pin":
            assert got == printed


@pytest.mark.parametrize("slices", [1, 2, 7, 33, 1000, 100000])
def test_count_any_slicing(slices):
    """The result does not depend on how many slices the lex order is cut
    into, including more slices than leaves."""
    for n, g in [(900, (13, 37, 38, 40)), (300, (11, 13, 17, 19, 23)), (77, (5, 9)),
                 (50, (3,)), (400, (29, 23, 19, 17, 13, 11))]:
        expect = oracle.count_dp(n, g)
        for method in (fs.METHOD_PAIR, fs.METHOD_PLAIN):
            cfg = fs.make_config(method=method, slices=slices)
            assert fs.fs_count(n, g, cfg) == expect, (n, g, slices, method)


def test_count_async_matches_sync():
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    for n, g in [workloads.CONFIG1, (2000, (13, 37, 38, 40, 41, 42))]:
        fs.fs_count_async(n, g, out[1:])
        torch.cuda.synchronize()
        assert int(out[1]) == oracle.count_dp(n, g)


def test_count_blocks_and_threads():
    n, g = 1500, (13, 37, 38, 40, 41, 42)
    expect = oracle.count_dp(n, g)
    for bt in (32, 64, 128, 256):
        for bps in (1, 2):
            cfg = fs.make_config(block_threads=bt, blocks_per_sm=bps)
            assert fs.fs_count(n, g, cfg) == expect


# ---------------------------------------------------------------------------
# length statistics
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("method", list(CONFIGS))
def test_length_stats_random(method):
    cfg = CONFIGS[method]
    for n, g in medium_cases():
        hl = oracle.hist_len(n, g)
        hist = torch.full((hl + 3,), 12345, dtype=torch.int64, device="cuda")
        cnt, mn, mx = fs.fs_length_stats(n, g, hist, cfg)
        ref = oracle.length_dp(n, g)
        mm = oracle.minmax_dp(n, g)
        assert cnt == int(ref.sum()), (n, g)
        if mm is None:
            assert (cnt, mn, mx) == (0, 0, 0)
        else:
            assert (mn, mx) == mm, (n, g)
        h = hist.cpu().numpy()
        assert np.array_equal(h[:hl].astype(np.uint64), ref), (n, g)
        assert np.all(h[hl:] == 12345)  # nothing written past the bins


def test_length_stats_config1():
    n, g = workloads.CONFIG1
    hist = torch.zeros(oracle.hist_len(n, g), dtype=torch.int64, device="cuda")
    assert fs.fs_length_stats(n, g, hist) == (4627, 40, 100)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), oracle.length_dp(n, g))


# ---------------------------------------------------------------------------
# any (predicate consumer)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("method", ["pair", "plain"])
def test_any_random_predicates(method):
    cfg = CONFIGS[method]
    rng = np.random.default_rng(17)
    cases = [(n, g) for n, g in medium_cases() if n <= 200]
    for n, g in cases:
        rows = oracle.brute(n, g) if len(g) <= 4 and n <= 120 else oracle.enumerate_sorted(n, g)
        d = len(g)
        for _ in range(6):
            w = [int(x) for x in rng.integers(-4, 5, size=d)]
            op = int(rng.integers(0, 3))
            modulus = int(rng.choice([0, 0, 0, 2, 5, 9]))
            if rows.shape[0] and rng.random() < 0.5:
                # aim at a value that occurs
                r = rows[int(rng.integers(0, rows.shape[0]))].astype(np.int64)
                c = int(np.dot(r, np.asarray(w, dtype=np.int64))) + int(rng.integers(-1, 2))
            else:
                c = int(rng.integers(-30, 60))
            expect = bool(oracle.pred_holds_rows(rows, w, c, op, modulus).any()) if rows.shape[0] else False
            assert fs.fs_any(n, g, w, c, op, modulus, cfg) == expect, (n, g, w, c, op, modulus)
            assert oracle.any_pred(n, g, w, c, op, modulus) == expect


def test_any_length_equals_histogram_support():
    n, g = workloads.CONFIG1
    hist = oracle.length_dp(n, g)
    for L in range(30, 110):
        assert fs.fs_any(n, g, [1] * 4, L, 0) == (L < len(hist) and hist[L] > 0)


def test_any_uses_generator():
    """'uses generator i' (w = e_i, >= 1) and its negation."""
    n, g = 300, (11, 13, 17, 19)
    rows = oracle.enumerate_sorted(n, g)
    for i in range(4):
        w = [0] * 4
        w[i] = 1
        assert fs.fs_any(n, g, w, 1, 2) == bool((rows[:, i] >= 1).any())
        assert fs.fs_any(n, g, w, 0, 0) == bool((rows[:, i] == 0).any())


# ---------------------------------------------------------------------------
# enumerate
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("method", list(CONFIGS))
def test_enumerate_random_sets(method):
    cfg = CONFIGS[method]
    for n, g in medium_cases():
        ref = oracle.enumerate_sorted(n, g)
        cnt, out = gpu_enumerate(n, g, cfg, extra_rows=3)
        d = len(g)
        assert cnt == ref.shape[0], (n, g)
        rows = out[:cnt * d].view(-1, d).cpu().numpy() if cnt else np.zeros((0, d), np.int32)
        assert np.array_equal(lexsort_rows(rows), ref), (n, g)
        # nothing past the last row was touched
        assert torch.all(out[cnt * d:] == -7)


@pytest.mark.parametrize("method", ["pair_keep", "plain_keep"])
def test_enumerate_order_keep_order_is_lex_ascending(method):
    """With the caller's generator order the buffer IS the oracle's
    lex-ascending list, byte for byte."""
    for n, g in medium_cases():
        ref = oracle.enumerate_sorted(n, g)
        cnt, out = gpu_enumerate(n, g, CONFIGS[method])
        d = len(g)
        rows = out[:cnt * d].view(-1, d).cpu().numpy() if cnt else np.zeros((0, d), np.int32)
        assert np.array_equal(rows, ref), (n, g)


def test_enumerate_plain_and_pair_buffers_identical():
    for n, g in medium_cases()[:30]:
        c1, o1 = gpu_enumerate(n, g, PAIR)
        c2, o2 = gpu_enumerate(n, g, PLAIN)
        assert c1 == c2
        assert torch.equal(o1[:c1 * len(g)], o2[:c2 * len(g)])


def test_enumerate_int16():
    for n, g in [workloads.CONFIG1, (2000, (13, 37, 38, 40, 41, 42)), (300, (1, 2, 3))]:
        ref = oracle.enumerate_sorted(n, g)
        cnt, out = gpu_enumerate(n, g, elem_bytes=2)
        rows = out[:cnt * len(g)].view(-1, len(g)).cpu().numpy().astype(np.int32)
        assert np.array_equal(lexsort_rows(rows), ref)


def test_enumerate_capacity():
    n, g = workloads.CONFIG1
    ref_count = 4627
    for cap in (0, 1, 5, 100, 4626):
        d = len(g)
        out = torch.full((cap * d + 64,), -7, dtype=torch.int32, device="cuda")
        with pytest.raises(fs.FsError) as e:
            fs.fs_enumerate(n, g, out, cap=cap)
        assert e.value.status == fs.FS_E_CAPACITY
        cnt = fs.fs_enumerate(n, g, out, cap=cap, allow_capacity=True)
        assert cnt == ref_count
        assert torch.all(out[cap * d:] == -7)  # nothing written past cap rows
    # the first cap rows are the first cap rows of the full buffer
    full_cnt, full = gpu_enumerate(n, g)
    out = torch.full((100 * 4,), -7, dtype=torch.int32, device="cuda")
    fs.fs_enumerate(n, g, out, cap=100, allow_capacity=True)
    assert torch.equal(out, full[:400])


def test_enumerate_async_matches_sync():
    n, g = 2000, (13, 37, 38, 40, 41, 42)
    cnt, ref = gpu_enumerate(n, g)
    out = torch.zeros_like(ref)
    dc = torch.zeros(1, dtype=torch.int64, device="cuda")
    fs.fs_enumerate_async(n, g, out, cnt, dc)
    torch.cuda.synchronize()
    assert int(dc[0]) == cnt
    assert torch.equal(out[:cnt * 6], ref[:cnt * 6])


def test_enumerate_big_leaves():
    """Leaves with very many rows (the last two generators small, n large)."""
    for n, g in [(4000, (1000, 1, 1)), (3000, (2, 1)), (20000, (7000, 3, 2)), (5000, (1, 1))]:
        expect = oracle.count_dp(n, g)
        cnt, out = gpu_enumerate(n, g)
        assert cnt == expect
        rows = out[:cnt * len(g)].view(-1, len(g)).cpu().numpy().astype(np.int64)
        assert np.all(rows @ np.asarray(g, dtype=np.int64) == n)
        assert np.unique(rows, axis=0).shape[0] == cnt


# ---------------------------------------------------------------------------
# slices (Sec. 4)
# ---------------------------------------------------------------------------

def walk_gens(g, order):
    return [g[i] for i in order]


@pytest.mark.parametrize("slices", [1, 2, 7, 64, 1000, 5000])
def test_plan_and_slice_counts_match_oracle(slices):
    """Every planner slice [B_s, B_{s+1}) holds exactly the factorizations the
    oracle's bounded stream finds between those bounds; the slices are
    disjoint, cover Z, and are balanced in leaves."""
    for n, g in [(600, (13, 37, 38, 40)), (200, (11, 13, 17, 19, 23)), (300, (7, 5, 3)),
                 workloads.CONFIG1]:
        order, bounds, leaves = fs.fs_plan(n, g, slices, PAIR)
        wg = walk_gens(g, order)
        for method in (fs.METHOD_PAIR, fs.METHOD_PLAIN):
            counts = fs.fs_slice_counts(n, g, slices, fs.make_config(method=method))
            total = 0
            for s in range(slices):
                lo = bounds[s]
                if lo[0] < 0:
                    assert counts[s] == 0
                    continue
                hi = bounds[s + 1] if bounds[s + 1][0] >= 0 else None
                c, _, _, _, _ = oracle.range_stats(n, wg, lo, hi, with_hist=False)
                assert counts[s] == c, (n, g, s)
                total += c
            assert total == oracle.count_dp(n, g)
        # bounds are clean prefixes (leaf, 0, 0) with phi <= n, non-decreasing
        # (an empty slice repeats the next slice's bound), min(S, L) distinct
        live = [b for b in bounds[:-1] if b[0] >= 0]
        for b in live:
            assert b[-1] == 0 and (len(b) < 3 or b[-2] == 0)
            assert sum(x * y for x, y in zip(b, wg)) <= n
        assert all(tuple(a) <= tuple(b) for a, b in zip(live, live[1:]))
        assert len(set(map(tuple, live))) == min(slices, leaves)
        if slices <= leaves:
            assert len(live) == slices


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("slices", [1, 3, 64, 2000])
def test_triple_slices_match_oracle(slices, k):
    """Trailing-k slices cut the prefixes k - 2 levels shorter; each slice
    still holds exactly what the oracle's bounded stream finds between its
    bounds."""
    cfg = TRIPLE if k == 3 else QUAD
    cases = [(600, (13, 37, 38, 40)), (250, (11, 13, 17, 19, 23)), workloads.CONFIG1,
             (700, (5, 7, 9, 11, 13, 15))]
    for n, g in cases:
        if len(g) < k + 1:
            continue
        order, bounds, leaves = fs.fs_plan(n, g, slices, cfg)
        counts = fs.fs_slice_counts(n, g, slices, cfg)
        wg = walk_gens(g, order)
        total = 0
        for s_ in range(slices):
            lo = bounds[s_]
            if lo[0] < 0:
                assert counts[s_] == 0
                continue
            assert all(x == 0 for x in lo[-k:])
            hi = bounds[s_ + 1] if bounds[s_ + 1][0] >= 0 else None
            c, _, _, _, _ = oracle.range_stats(n, wg, lo, hi, with_hist=False)
            assert counts[s_] == c, (n, g, s_)
            total += c
        assert total == oracle.count_dp(n, g)


def test_enumerate_slices_sampled_against_oracle_stream():
    """Rows of sampled slices equal the oracle's bounded stream for the same
    bounds (reversed to ascending), at their scanned offsets."""
    n, g = 1200, (13, 37, 38, 40, 41)
    S = 257
    cfg = fs.make_config(method=fs.METHOD_PAIR, slices=S)
    order, bounds, _ = fs.fs_plan(n, g, S, cfg)
    counts = fs.fs_slice_counts(n, g, S, cfg)
    offs = np.concatenate([[0], np.cumsum(counts)])
    cnt, out = gpu_enumerate(n, g, cfg)
    d = len(g)
    rows = out[:cnt * d].view(-1, d).cpu().numpy()
    wg = walk_gens(g, order)
    rng = np.random.default_rng(3)
    for s in rng.choice(S, 25, replace=False):
        lo = bounds[s]
        if lo[0] < 0:
            continue
        hi = bounds[s + 1] if bounds[s + 1][0] >= 0 else None
        ref, _ = oracle.enumerate_range(n, wg, lo, hi)
        ref = ref[::-1]
        got = rows[offs[s]:offs[s + 1]][:, order]  # to walk order
        assert np.array_equal(got, ref), s


# ---------------------------------------------------------------------------
# the benchmark workloads at full size
# ---------------------------------------------------------------------------

def test_config2_full():
    """g=(11,13,17,19,23,29), n=3000: count, length statistics, and the full
    1.73 GB enumeration (every row sums to n, rows strictly ascending in the
    walk order -- hence distinct -- and as many as the exact count, so the set
    is Z), plus sampled slices compared row for row with the oracle."""
    n, g = workloads.CONFIG2
    expect = oracle.count_dp(n, g)
    assert expect == 72082790
    assert fs.fs_count(n, g) == expect
    hist = torch.zeros(oracle.hist_len(n, g), dtype=torch.int64, device="cuda")
    assert fs.fs_length_stats(n, g, hist) == (expect, 104, 272)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), oracle.length_dp(n, g))
    d = len(g)
    S = 4096
    cfg = fs.make_config(method=fs.METHOD_PAIR, slices=S)
    out = torch.empty(expect * d, dtype=torch.int32, device="cuda")
    assert fs.fs_enumerate(n, g, out, cfg=cfg) == expect
    rows = out.view(-1, d)
    gv = torch.tensor(g, dtype=torch.int64, device="cuda")
    order, bounds, _ = fs.fs_plan(n, g, S, cfg)
    key = torch.zeros(expect, dtype=torch.int64, device="cuda")
    for k in order:  # walk order, most significant first; coordinates < 512
        key = key * 512 + rows[:, k].to(torch.int64)
    for c0 in range(0, expect, 1 << 24):
        blk = rows[c0:c0 + (1 << 24)].to(torch.int64)
        assert bool(torch.all((blk * gv).sum(dim=1) == n))
        assert bool(torch.all(blk >= 0))
    assert bool(torch.all(key[1:] > key[:-1]))
    counts = fs.fs_slice_counts(n, g, S, cfg)
    offs = np.concatenate([[0], np.cumsum(counts)])
    wg = walk_gens(g, order)
    rng = np.random.default_rng(5)
    for s in list(rng.choice(S, 6, replace=False)) + [0, S - 1]:
        lo = bounds[s]
        hi = bounds[s + 1] if bounds[s + 1][0] >= 0 else None
        ref, _ = oracle.enumerate_range(n, wg, lo, hi)
        got = rows[offs[s]:offs[s + 1]].cpu().numpy()[:, order]
        assert np.array_equal(got, ref[::-1]), s
    del out, rows, key
    torch.cuda.empty_cache()


def test_config3_count_and_lengths_dp_exact():
    """8 generators from seed 0, n = 40000: 7,655,692,813,487 factorizations.
    Count and the full length histogram equal the exact DP; sampled slices
    equal the oracle's bounded stream."""
    n, g = workloads.config3(0)
    expect = oracle.count_dp(n, g)
    assert expect == 7655692813487
    assert fs.fs_count(n, g) == expect
    hist = torch.zeros(oracle.hist_len(n, g), dtype=torch.int64, device="cuda")
    cnt, mn, mx = fs.fs_length_stats(n, g, hist)
    ref = oracle.length_dp(n, g)
    assert cnt == expect
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), ref)
    assert (mn, mx) == oracle.minmax_dp(n, g)
    assert fs.fs_count(n, g, PAIR) == expect
    assert fs.fs_count(n, g, TRIPLE) == expect
    assert fs.fs_count(n, g, QUAD) == expect
    assert fs.fs_length_stats(n, g, None) == (expect,) + oracle.minmax_dp(n, g)
    assert fs.fs_length_stats(n, g, None, TRIPLE) == (expect,) + oracle.minmax_dp(n, g)
    S = 1 << 20
    order, bounds, leaves = fs.fs_plan(n, g, S, PAIR)
    counts = fs.fs_slice_counts(n, g, S, PAIR)
    assert sum(counts) == expect
    wg = walk_gens(g, order)
    rng = np.random.default_rng(9)
    for s in rng.choice(S, 3, replace=False):
        hi = bounds[s + 1] if bounds[s + 1][0] >= 0 else None
        c, _, _, _, _ = oracle.range_stats(n, wg, bounds[s], hi, with_hist=False)
        assert counts[s] == c, s


@pytest.mark.parametrize("seed", [1, 2])
def test_config3_other_seeds(seed):
    n, g = workloads.config3(seed)
    expect = oracle.count_dp(n, g)
    assert fs.fs_count(n, g) == expect
    assert fs.fs_count(n, g, PAIR) == expect
    assert fs.fs_count(n, g, TRIPLE) == expect
    # the length range from the trailing tables (count walk, then range walk)
    assert fs.fs_length_stats(n, g, None) == (expect,) + oracle.minmax_dp(n, g)


# ---------------------------------------------------------------------------
# common-divisor skipping: generators that share divisors
# ---------------------------------------------------------------------------
DIVISOR_CASES = [(97, (6, 10)), (240, (6, 10, 15)), (401, (4, 6, 8, 10)), (300, (12, 18, 27, 8)),
                 (420, (30, 42, 70, 105, 11)), (513, (2, 4, 6, 8, 10)), (512, (2, 4, 6, 8, 10)),
                 (900, (35, 21, 15, 9, 25, 49)), (777, (14, 21, 6, 10, 15, 35)),
                 (1000, (100, 60, 36, 24, 18, 8, 12)), (250, (5, 10, 15, 20, 25, 30)),
                 (330, (22, 33, 55, 9, 6, 4))]


@pytest.mark.parametrize("cfg", [PAIR, PAIR_KEEP, TRIPLE, QUAD, AUTO],
                         ids=["pair", "pair_keep", "triple", "quad", "auto"])
def test_common_divisor_counts_and_lengths(cfg):
    """Walks that skip the leaves (and runs) whose residual cannot be a
    multiple of the trailing generators' gcd give the exact counts and
    length ranges."""
    dmin = {id(TRIPLE): 4, id(QUAD): 5}.get(id(cfg), 1)
    for n, g in DIVISOR_CASES:
        if len(g) < dmin:
            continue
        assert fs.fs_count(n, g, cfg) == oracle.count_dp(n, g), (n, g)
        mm = oracle.minmax_dp(n, g) or (0, 0)
        assert fs.fs_length_stats(n, g, None, cfg) == (oracle.count_dp(n, g),) + tuple(mm), (n, g)


@pytest.mark.parametrize("method", ["pair", "pair_keep"])
def test_common_divisor_enumerate_histogram_any(method):
    cfg = CONFIGS[method]
    for n, g in DIVISOR_CASES:
        rows = oracle.enumerate_sorted(n, g)
        got, out = gpu_enumerate(n, g, cfg)
        assert got == rows.shape[0]
        d = len(g)
        mine = out[:got * d].view(got, d).cpu().numpy() if got else np.zeros((0, d), np.int32)
        if method == "pair_keep":
            assert np.array_equal(mine, rows), (n, g)  # lex-ascending in the caller's order
        else:
            assert np.array_equal(lexsort_rows(mine), rows), (n, g)
        hist = torch.zeros(oracle.hist_len(n, g), dtype=torch.int64, device="cuda")
        fs.fs_length_stats(n, g, hist, cfg)
        assert np.array_equal(hist.cpu().numpy().astype(np.uint64), oracle.length_dp(n, g)), (n, g)
        w = [1] * d
        for L in range(0, oracle.hist_len(n, g), 7):
            assert fs.fs_any(n, g, w, L, cfg=cfg) == oracle.any_pred(n, g, w, L), (n, g, L)


def test_common_divisor_slices_and_plain_agree():
    """Per-slice counts with skipping equal the oracle's bounded streams, and
    the PLAIN walk (no skipping) gives the same buffers."""
    for n, g in DIVISOR_CASES[:6]:
        for slices in (1, 5, 300):
            order, bounds, leaves = fs.fs_plan(n, g, slices, PAIR)
            counts = fs.fs_slice_counts(n, g, slices, PAIR)
            wg = walk_gens(g, order)
            for s_ in range(slices):
                lo = bounds[s_]
                if lo[0] < 0:
                    assert counts[s_] == 0
                    continue
                hi = bounds[s_ + 1] if bounds[s_ + 1][0] >= 0 else None
                c, _, _, _, _ = oracle.range_stats(n, wg, lo, hi, with_hist=False)
                assert counts[s_] == c, (n, g, slices, s_)
        a, oa = gpu_enumerate(n, g, PAIR)
        b, ob = gpu_enumerate(n, g, PLAIN)
        assert a == b and torch.equal(oa[:a * len(g)], ob[:b * len(g)])
