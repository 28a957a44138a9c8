"""Batched queries (many (n, g) in one persistent launch) against the oracle:
exact counts and min / max lengths per query, invalid queries flagged and
skipped, the same results under every launch shape the autotuner tries, and
under CUDA-graph replay."""
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


def expected(queries, mode):
    out = []
    for n, g in queries:
        c = oracle.count_dp(n, g)
        mm = oracle.minmax_dp(n, g) if mode == fs.BATCH_LENGTHS else None
        if mm is None:
            mm = (0, 0)
        out.append((c, mm[0], mm[1], fs.FS_OK))
    return out


@pytest.mark.parametrize("mode", [fs.BATCH_COUNT, fs.BATCH_LENGTHS])
def test_batch_small_random(mode):
    qs = workloads.config4(seed=3, nq=300, n_max=1500)
    qs += [(0, (3, 5, 7)), (17, (5,)), (10, (5, 5)), (97, (1, 1, 1)), (7, (4, 6)),
           (500, (5, 7, 11, 13)), (1000, (13, 37, 38))]
    got = fs.fs_batch_run(qs, mode)
    assert got == expected(qs, mode)


@pytest.mark.parametrize("method", [fs.METHOD_PAIR, fs.METHOD_TRIPLE, fs.METHOD_QUAD])
def test_batch_methods_agree(method):
    """Pair walks, trailing-three and trailing-four tables give the same
    per-query results."""
    qs = workloads.config4(seed=13, nq=200, n_max=4000)
    cfg = fs.make_config(method=method)
    assert fs.fs_batch_run(qs, fs.BATCH_LENGTHS, cfg) == expected(qs, fs.BATCH_LENGTHS)


def test_batch_invalid_queries_are_flagged_and_skipped():
    qs = [(100, (3, 5, 7)), (100, (3, 0, 7)), (-5, (2, 3)), (2**31 - 3, (5, 7, 9)),
          (200, (11, 13))]
    got = fs.fs_batch_run(qs, fs.BATCH_LENGTHS)
    assert got[0][:3] == (oracle.count_dp(100, (3, 5, 7)),) + oracle.minmax_dp(100, (3, 5, 7))
    assert got[1][3] == fs.FS_E_INVAL and got[1][0] == 0
    assert got[2][3] == fs.FS_E_INVAL and got[2][0] == 0
    assert got[3][3] == fs.FS_E_OVERFLOW and got[3][0] == 0
    mm = oracle.minmax_dp(200, (11, 13))
    assert got[4] == (oracle.count_dp(200, (11, 13)), mm[0], mm[1], fs.FS_OK)


def test_batch_config4_full():
    """4096 seeded queries: d in [3, 8], distinct generators in [5, 100], n in
    [100, 5000]; every count and min / max length equals the oracle's."""
    qs = workloads.config4(seed=0)
    got = fs.fs_batch_run(qs, fs.BATCH_LENGTHS)
    assert got == expected(qs, fs.BATCH_LENGTHS)
    # and the count-only mode agrees
    got0 = fs.fs_batch_run(qs, fs.BATCH_COUNT)
    assert [g[0] for g in got0] == [g[0] for g in got]


def test_batch_same_results_under_every_shape():
    qs = workloads.config4(seed=5, nq=200, n_max=2500)
    ref = expected(qs, fs.BATCH_LENGTHS)
    for bt in (64, 128, 256):
        for items in (1, 7, 500, 100000):
            cfg = fs.make_config(block_threads=bt, slices=items)
            assert fs.fs_batch_run(qs, fs.BATCH_LENGTHS, cfg) == ref, (bt, items)
    best, ms = fs.fs_batch_autotune(qs, fs.BATCH_LENGTHS)
    assert ms > 0 and best.block_threads in (128, 256)
    assert fs.fs_batch_run(qs, fs.BATCH_LENGTHS, best) == ref


def test_batch_handle_relaunch_and_graph_replay():
    qs = workloads.config4(seed=9, nq=128, n_max=2000)
    ref = expected(qs, fs.BATCH_LENGTHS)
    with fs.Batch(qs, fs.BATCH_LENGTHS) as b:
        b.launch()
        assert b.results() == ref
        b.launch()
        b.launch()
        assert b.results() == ref
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            b.launch(stream=s.cuda_stream)  # warm-up outside capture
            s.synchronize()
            with torch.cuda.graph(g, stream=s):
                b.launch(stream=s.cuda_stream)
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        assert b.results() == ref


def test_batch_matches_single_query_calls():
    qs = workloads.config4(seed=11, nq=64, n_max=3000)
    got = fs.fs_batch_run(qs, fs.BATCH_LENGTHS)
    for (n, g), r in zip(qs, got):
        assert fs.fs_length_stats(n, g) == r[:3]


@pytest.mark.parametrize("method", [fs.METHOD_PAIR, fs.METHOD_AUTO])
def test_batch_common_divisors(method):
    """Queries whose generators share divisors (the walks skip leaves and runs
    that cannot complete) against the oracle."""
    qs = [(97, (6, 10)), (240, (6, 10, 15)), (401, (4, 6, 8, 10)), (300, (12, 18, 27, 8)),
          (420, (30, 42, 70, 105, 11)), (513, (2, 4, 6, 8, 10)), (512, (2, 4, 6, 8, 10)),
          (900, (35, 21, 15, 9, 25, 49)), (1000, (100, 60, 36, 24, 18, 8, 12)),
          (3000, (14, 21, 6, 10, 15, 35))]
    cfg = fs.make_config(method=method)
    assert fs.fs_batch_run(qs, fs.BATCH_LENGTHS, cfg) == expected(qs, fs.BATCH_LENGTHS)


def test_batch_slot_switches_mode_between_loads():
    """One slot reserved for length ranges serves count-only loads (count mode,
    no length tables) and length loads in turn, each exact."""
    qs = workloads.config4(seed=13, nq=96, n_max=3000)
    with fs.BatchSlot(128, 256 << 20, fs.BATCH_LENGTHS) as b:
        for mode in (fs.BATCH_COUNT, fs.BATCH_LENGTHS, fs.BATCH_COUNT):
            b.load(qs, mode)
            b.launch()
            assert b.results() == expected(qs, mode), mode
        with pytest.raises(fs.FsError):
            b.load(qs, 7)
