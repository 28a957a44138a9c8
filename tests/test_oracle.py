"""Pins for the CPU oracle: it is checked against what the paper and the
mathematics fix, never against itself or the CUDA path.

* Table 1 (Sec. 5.2): the printed |Z(n)| column.
* The definition of Z (Sec. 1) by brute force on tiny inputs.
* Closed forms: d = 1, d = 2 (textbook linear congruence), n = 0, repeated
  generators.
* Invariants of the stream (Thm 3.2, Thm 3.3): every output sums to n, strictly
  lex-decreasing, no duplicates, count equal to the generating-function DP.
* A closed form for the number of candidates Algorithm 3.1 produces.
* Slices (Sec. 4): any partition of the lex order by bounds gives disjoint
  slices whose union is the whole set.
* Mutation tests: each deliberately wrong variant of a step fails some pin.
"""
import os
from math import gcd

import numpy as np
import pytest

import oracle
from paper_2405_07989_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_counts.txt")


def table1_cells():
    cells = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            gens, n, printed, status = line.split()
            cells.append((tuple(int(x) for x in gens.split(",")), int(n), int(printed), status))
    return cells


def prefix_counts_below(n, gens):
    """#{(a_1..a_i) >= 0 : sum a_j g_j <= n - 1} for i = 1..d-1, by counting
    lattice points directly (numpy running sums, not the oracle)."""
    out = []
    if n <= 0:
        return [0] * (len(gens) - 1)
    for i in range(1, len(gens)):
        c = np.zeros(n, dtype=object)
        c[0] = 1
        for g in gens[:i]:
            for p in range(g, n):
                c[p] += c[p - g]
        out.append(int(sum(c)))
    return out


# --------------------------------------------------------------------------
# Table 1
# --------------------------------------------------------------------------

@pytest.mark.parametrize("cell", table1_cells(), ids=lambda c: f"{len(c[0])}-{c[1]}")
def test_table1_count_dp(cell):
    gens, n, printed, status = cell
    exact = oracle.count_dp(n, gens)
    if status == "pin":
        assert exact == printed
    else:
        # errata: the printed value is not the exact count
        assert exact != printed


@pytest.mark.parametrize("cell", [c for c in table1_cells() if c[1] <= 20000 and len(c[0]) <= 4
                                  or (len(c[0]) >= 5 and c[1] <= 2000)],
                         ids=lambda c: f"{len(c[0])}-{c[1]}")
def test_table1_stream(cell):
    """The paper's own algorithm (Algorithm 3.1 stream) reproduces Table 1."""
    gens, n, printed, status = cell
    cnt, _, _, _, _ = oracle.range_stats(n, gens, with_hist=False)
    if status == "pin":
        assert cnt == printed
    else:
        assert cnt == oracle.count_dp(n, gens) != printed


def test_table1_errata_by_stream():
    """The three errata cells: the stream and the DP agree with each other and
    both disagree with the printed value."""
    for gens, n, printed, status in table1_cells():
        if status != "errata" or n > 3000:
            continue
        cnt, _, _, _, _ = oracle.range_stats(n, gens, with_hist=False)
        assert cnt == oracle.count_dp(n, gens)
        assert cnt != printed


# --------------------------------------------------------------------------
# brute force, closed forms, special cases
# --------------------------------------------------------------------------

def test_stream_equals_brute_force_random_tiny():
    for n, gens in workloads.random_small(seed=1, count=400):
        a = oracle.enumerate_sorted(n, gens)
        b = oracle.brute(n, gens)
        assert a.shape == b.shape, (n, gens)
        assert np.array_equal(a, b), (n, gens)


def test_d1_closed_form():
    for g in (1, 2, 3, 7, 13):
        for n in range(0, 60):
            rows = oracle.enumerate_sorted(n, [g])
            if n % g == 0:
                assert rows.tolist() == [[n // g]]
            else:
                assert rows.shape[0] == 0


def test_d2_congruence_count():
    """|Z(n,(g,h))| = 0 unless G = gcd(g,h) divides n; else the number of
    a in [0, n/g] with a == (n/G) (g/G)^-1 (mod h/G)."""
    rng = np.random.default_rng(7)
    for _ in range(300):
        g, h = (int(x) for x in rng.integers(1, 40, size=2))
        n = int(rng.integers(0, 600))
        G = gcd(g, h)
        if n % G:
            expect = 0
        else:
            m = h // G
            a0 = ((n // G) * pow(g // G, -1, m)) % m if m > 1 else 0
            expect = 0 if a0 > n // g else (n // g - a0) // m + 1
        assert oracle.enumerate_sorted(n, [g, h]).shape[0] == expect
        assert oracle.count_dp(n, [g, h]) == expect


def test_n_zero_gives_origin():
    for d in range(1, 9):
        rows = oracle.enumerate_sorted(0, list(range(2, 2 + d)))
        assert rows.tolist() == [[0] * d]
        assert oracle.count_dp(0, list(range(2, 2 + d))) == 1


def test_repeated_generators():
    rows = oracle.enumerate_sorted(10, [5, 5])
    assert rows.tolist() == [[0, 2], [1, 1], [2, 0]]


# --------------------------------------------------------------------------
# stream invariants, DPs, candidate count
# --------------------------------------------------------------------------

INVARIANT_CASES = [
    workloads.CONFIG1,
    (200, (3, 5, 7)),
    (157, (4, 6, 9, 10)),
    (333, (23, 5, 17, 5, 11)),
    (90, (2, 3, 5, 7, 11, 13)),
    (1000, (13, 37, 38)),
]


@pytest.mark.parametrize("case", INVARIANT_CASES, ids=str)
def test_stream_invariants(case):
    n, gens = case
    rows, _ = oracle.enumerate_stream(n, gens)
    g = np.asarray(gens, dtype=np.int64)
    assert np.all(rows.astype(np.int64) @ g == n)
    assert np.all(rows >= 0)
    # strictly lex-decreasing: consecutive rows differ and the first
    # differing coordinate decreases
    for a, b in zip(rows[:-1], rows[1:]):
        k = np.nonzero(a != b)[0]
        assert k.size > 0 and a[k[0]] > b[k[0]]
    assert rows.shape[0] == oracle.count_dp(n, gens)


@pytest.mark.parametrize("case", INVARIANT_CASES, ids=str)
def test_length_statistics_vs_stream(case):
    n, gens = case
    cnt, mn, mx, hist, _ = oracle.range_stats(n, gens)
    rows = oracle.brute(n, gens)
    lens = rows.astype(np.int64).sum(axis=1)
    ref = np.bincount(lens, minlength=oracle.hist_len(n, gens)).astype(np.uint64)
    assert np.array_equal(hist, ref)
    assert np.array_equal(oracle.length_dp(n, gens), ref)
    assert int(hist.sum()) == cnt
    assert (mn, mx) == (int(lens.min()), int(lens.max()))
    assert oracle.minmax_dp(n, gens) == (mn, mx)


def test_minmax_dp_empty():
    assert oracle.minmax_dp(7, [4, 6]) is None
    cnt, mn, mx, hist, _ = oracle.range_stats(7, [4, 6])
    assert (cnt, mn, mx) == (0, 0, 0) and int(hist.sum()) == 0


@pytest.mark.parametrize("case", INVARIANT_CASES + [(0, (3, 4)), (17, (5,)), (40, (40, 1))],
                         ids=str)
def test_candidate_count_closed_form(case):
    """Algorithm 3.1 emits the first candidate, then exactly one candidate per
    prefix (a_1..a_i), 1 <= i <= d-1, with sum a_j g_j <= n - 1: the one where
    a_i was just decremented and a_{i+1} solved."""
    n, gens = case
    _, cand = oracle.enumerate_stream(n, gens)
    assert cand == 1 + sum(prefix_counts_below(n, gens))


def test_config_values():
    """Exact sizes of the two small benchmark workloads (count, length range)."""
    n, g = workloads.CONFIG1
    assert oracle.count_dp(n, g) == 4627
    assert oracle.minmax_dp(n, g) == (40, 100)
    assert np.array_equal(oracle.enumerate_sorted(n, g), oracle.brute(n, g))
    n, g = workloads.CONFIG2
    assert oracle.count_dp(n, g) == 72082790
    assert oracle.minmax_dp(n, g) == (104, 272)
    h = oracle.length_dp(n, g)
    assert int(h.sum()) == 72082790
    nz = np.nonzero(h)[0]
    assert (int(nz[0]), int(nz[-1])) == (104, 272)


# --------------------------------------------------------------------------
# slices (Sec. 4)
# --------------------------------------------------------------------------

def random_bounds(rng, n, gens, k):
    """k random bound vectors with last coordinate 0 and phi <= n (the
    hypothesis of Thm 3.2 / Remark 4.2 for a slice start), sorted, distinct."""
    d = len(gens)
    out = set()
    while len(out) < k:
        a = [0] * d
        left = n
        for j in range(d - 1):
            a[j] = int(rng.integers(0, left // gens[j] + 1))
            left -= a[j] * gens[j]
        out.add(tuple(a))
    return sorted(out)


@pytest.mark.parametrize("case", INVARIANT_CASES[:5], ids=str)
def test_slices_partition_the_set(case):
    n, gens = case
    rng = np.random.default_rng(11)
    full = oracle.enumerate_sorted(n, gens)
    for k in (1, 2, 7, 40):
        bounds = random_bounds(rng, n, gens, k)
        edges = [None] + bounds + [None]
        parts = []
        for lo, hi in zip(edges[:-1], edges[1:]):
            rows, _ = oracle.enumerate_range(n, gens, lo, hi)
            for r in rows:
                if lo is not None:
                    assert tuple(r) >= lo
                if hi is not None:
                    assert tuple(r) < hi
            cnt, _, _, _, _ = oracle.range_stats(n, gens, lo, hi, with_hist=False)
            assert cnt == rows.shape[0]
            parts.append(rows)
        allrows = np.concatenate([p[::-1] for p in parts])
        assert np.array_equal(allrows, full)


# --------------------------------------------------------------------------
# predicate consumer
# --------------------------------------------------------------------------

def test_any_vs_explicit_rows():
    rng = np.random.default_rng(5)
    for n, gens in workloads.random_small(seed=3, count=200, d_max=5, n_max=80):
        rows = oracle.brute(n, gens)
        d = len(gens)
        w = [int(x) for x in rng.integers(-3, 4, size=d)]
        op = int(rng.integers(0, 3))
        modulus = int(rng.choice([0, 0, 3, 7]))
        c = int(rng.integers(-10, 40))
        expect = bool(oracle.pred_holds_rows(rows, w, c, op, modulus).any()) if len(rows) else False
        assert oracle.any_pred(n, gens, w, c, op, modulus) == expect


def test_any_length_equals_histogram_support():
    n, g = workloads.CONFIG1
    hist = oracle.length_dp(n, g)
    for L in range(30, 110):
        assert oracle.any_pred(n, g, [1] * 4, L, 0) == (L < len(hist) and hist[L] > 0)


# --------------------------------------------------------------------------
# mutations: each planted mistake fails a pin
# --------------------------------------------------------------------------

def _pins_pass():
    for gens, n, printed, status in table1_cells():
        if status == "pin" and n <= 5000:
            cnt, _, _, _, _ = oracle.range_stats(n, gens, with_hist=False)
            if cnt != printed:
                return False
    for n, gens in workloads.random_small(seed=1, count=150):
        a = oracle.enumerate_sorted(n, gens)
        b = oracle.brute(n, gens)
        if a.shape != b.shape or not np.array_equal(a, b):
            return False
    for n, gens in INVARIANT_CASES[:4]:
        _, cand = oracle.enumerate_stream(n, gens)
        if cand != 1 + sum(prefix_counts_below(n, gens)):
            return False
    return True


@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5])
def test_planted_mistakes_are_caught(mutation):
    try:
        oracle.set_mutation(mutation)
        assert not _pins_pass()
    finally:
        oracle.set_mutation(0)
    assert _pins_pass()
