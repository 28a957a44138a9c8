"""The serving loop (fs_server_*): every response equals the oracle and the
single-query call made alone, whether the request ran alone or inside a mix
of counts, length statistics and enumerations arriving while other batches
are on the GPU; enumerations are admitted by their exact output bytes."""
import time

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


class _DevRows:
    """A device address seen as a tensor (no copy), through the CUDA array interface."""

    def __init__(self, ptr, rows, d, elem_bytes):
        self.__cuda_array_interface__ = {
            "shape": (rows, d), "typestr": "<i2" if elem_bytes == 2 else "<i4",
            "data": (ptr, False), "version": 3, "strides": None}


def hist_of(resp, n, g):
    """A LENGTHS response's histogram (hist=True), read from the device."""
    bins = n // min(g) + 1
    t = torch.as_tensor(_DevHist(resp["rows"], bins), device="cuda")
    return t.cpu().numpy().astype(np.uint64)


class _DevHist:
    def __init__(self, ptr, bins):
        self.__cuda_array_interface__ = {"shape": (bins,), "typestr": "<u8", "data": (ptr, False),
                                         "version": 3, "strides": None}


def rows_of(resp, d, elem_bytes):
    if resp["count"] == 0:
        return np.zeros((0, d), dtype=np.int64)
    t = torch.as_tensor(_DevRows(resp["rows"], resp["count"], d, elem_bytes), device="cuda")
    return t.cpu().numpy().astype(np.int64)


def alone(op, n, g, elem_bytes=2, keep_order=False):
    """The same request through the single-query entry points."""
    cfg = fs.make_config(keep_order=keep_order)
    if op == fs.REQ_COUNT:
        return (fs.fs_count(n, g),)
    if op == fs.REQ_LENGTHS:
        return fs.fs_length_stats(n, g)
    c = fs.fs_count(n, g)
    dt = torch.int16 if elem_bytes == 2 else torch.int32
    out = torch.empty((max(c, 1), len(g)), dtype=dt, device="cuda")
    fs.fs_enumerate(n, g, out, cap=c, elem_bytes=elem_bytes, cfg=cfg)
    return out[:c].cpu().numpy().astype(np.int64)


def drain(srv, tickets, timeout_s=120.0):
    got = {}
    t0 = time.time()
    while len(got) < len(tickets):
        for r in srv.poll(256, wait_ms=50):
            got[r["ticket"]] = r
        assert time.time() - t0 < timeout_s, f"{len(got)} of {len(tickets)} responses"
    return got


def check(resp, op, n, g, elem_bytes=2, keep_order=False, hist=False):
    assert resp["status"] == fs.FS_OK, resp
    c = oracle.count_dp(n, g)
    assert resp["count"] == c
    if op in (fs.REQ_LENGTHS, fs.REQ_ENUMERATE) and c > 0:
        assert (resp["min_len"], resp["max_len"]) == oracle.minmax_dp(n, g)
    job = op == fs.REQ_ENUMERATE or (op == fs.REQ_LENGTHS and hist)
    # a count or length request run as a job from the start (no batch) is
    # launched, counted and answered by its job
    direct = resp["t_job"] > 0 and resp["t_start"] == resp["t_job"]
    # the stages in order; a job's launch between the count and the answer
    assert resp["t_submit"] <= resp["t_start"] <= resp["t_counted"] <= resp["t_done"], resp
    if direct:
        assert op != fs.REQ_ENUMERATE and resp["t_counted"] <= resp["t_done"], resp
        assert (resp["rows"] != 0) == hist, resp
    elif job:
        assert resp["t_counted"] <= resp["t_job"] <= resp["t_done"], resp
    else:
        assert resp["t_job"] == 0.0 and resp["rows"] == 0, resp
    ref = alone(op, n, g, elem_bytes, keep_order)
    if op == fs.REQ_COUNT:
        assert (resp["count"],) == ref
    elif op == fs.REQ_LENGTHS:
        assert (resp["count"], resp["min_len"], resp["max_len"]) == ref
        if hist:  # bin for bin: the oracle's bivariate DP and the call alone
            h = hist_of(resp, n, g)
            assert np.array_equal(h, oracle.length_dp(n, g)), (n, g)
            alone_h = torch.zeros(n // min(g) + 1, dtype=torch.int64, device="cuda")
            fs.fs_length_stats(n, g, alone_h)
            assert np.array_equal(h, alone_h.cpu().numpy().astype(np.uint64))
    else:
        rows = rows_of(resp, len(g), elem_bytes)
        assert np.array_equal(rows, ref)  # byte-identical to the call alone
        if c <= 200000:  # and the same set as the oracle's
            srt = rows[np.lexsort(rows.T[::-1])] if c else rows
            assert np.array_equal(srt, oracle.enumerate_sorted(n, g).astype(np.int64).reshape(-1, len(g)))


def test_server_mix_matches_alone():
    """A config-5-like mix (80 % count, 15 % lengths, 5 % enumerate), submitted
    in bursts while earlier batches run."""
    reqs = workloads.config5(seed=4, nreq=240, n_max=2500)
    with fs.Server(mem_budget_bytes=512 << 20, max_batch=64, slots=3, window_us=100,
                   job_streams=3) as srv:
        tickets = {}
        for i, (_, op, n, g) in enumerate(reqs):
            hist = op == fs.REQ_LENGTHS and i % 2 == 0  # every other one with its histogram
            tickets[srv.submit(op, n, g, elem_bytes=2, hist=hist)] = (op, n, g, hist)
            if i % 40 == 39:
                time.sleep(0.002)
        got = drain(srv, tickets)
        assert sum(1 for op, _, _, h in tickets.values() if h) > 0
        for t, (op, n, g, hist) in tickets.items():
            check(got[t], op, n, g, hist=hist)
            if op == fs.REQ_ENUMERATE or hist:
                srv.release(t)


def test_server_jobs_run_concurrently():
    """Enumerations that fit the budget together run on the job streams at
    the same time: some two of them overlap between launch and completion
    (each writes about 2 GB of int16 rows), and each one's rows equal the
    call made alone, byte for byte (compared on the device)."""
    n, g = 3600, (11, 13, 17, 19, 23, 29)
    c = fs.fs_count(n, g)
    d = len(g)
    ref = torch.empty((c, d), dtype=torch.int16, device="cuda")
    fs.fs_enumerate(n, g, ref, cap=c, elem_bytes=2)
    with fs.Server(mem_budget_bytes=4 * c * d * 2 + (1 << 20), max_batch=16, job_streams=4) as srv:
        ts = [srv.submit(fs.REQ_ENUMERATE, n, g, elem_bytes=2) for _ in range(4)]
        got = drain(srv, ts)
        iv = sorted((got[t]["t_job"], got[t]["t_done"]) for t in ts)
        assert any(iv[i + 1][0] < iv[i][1] for i in range(len(iv) - 1)), iv
        for t in ts:
            assert got[t]["status"] == fs.FS_OK and got[t]["count"] == c
            rows = torch.as_tensor(_DevRows(got[t]["rows"], c, d, 2), device="cuda")
            assert torch.equal(rows, ref)
            srv.release(t)
    del ref
    torch.cuda.empty_cache()


@pytest.mark.parametrize("op,hist", [(fs.REQ_COUNT, False), (fs.REQ_LENGTHS, False),
                                     (fs.REQ_LENGTHS, True), (fs.REQ_ENUMERATE, False)])
def test_server_request_alone(op, hist):
    n, g = 2000, (11, 13, 17, 19, 23)
    with fs.Server(mem_budget_bytes=64 << 20) as srv:
        t = srv.submit(op, n, g, elem_bytes=4, keep_order=True, hist=hist)
        got = drain(srv, {t: None})
        check(got[t], op, n, g, elem_bytes=4, keep_order=True, hist=hist)
        if op == fs.REQ_ENUMERATE or hist:
            srv.release(t)


def test_server_invalid_and_capacity():
    n_big, g_big = 3000, (11, 13, 17, 19, 23, 29)  # 72 082 790 rows: 865 MB of int16
    with fs.Server(mem_budget_bytes=8 << 20, max_batch=16) as srv:
        ts = [srv.submit(fs.REQ_COUNT, 100, (3, 0, 7)),
              srv.submit(fs.REQ_ENUMERATE, n_big, g_big, elem_bytes=2),
              srv.submit(fs.REQ_LENGTHS, 700, (5, 7, 11, 13)),
              srv.submit(fs.REQ_ENUMERATE, 40000, (1, 2), elem_bytes=2)]  # a_1 up to 40000: no int16
        got = drain(srv, ts)
        assert got[ts[0]]["status"] == fs.FS_E_INVAL
        assert got[ts[1]]["status"] == fs.FS_E_CAPACITY
        assert got[ts[1]]["count"] == oracle.count_dp(n_big, g_big)
        check(got[ts[2]], fs.REQ_LENGTHS, 700, (5, 7, 11, 13))
        assert got[ts[3]]["status"] == fs.FS_E_OVERFLOW
        with pytest.raises(fs.FsError):
            srv.submit(7, 100, (3, 5))
        with pytest.raises(fs.FsError):
            srv.submit(fs.REQ_ENUMERATE, 100, (3, 5), elem_bytes=8)
        r = fs.fs_request()
        r.n, r.d, r.op, r.hist = 100, 2, fs.REQ_LENGTHS, 5
        r.gens[0], r.gens[1] = 3, 5
        t = fs.ctypes.c_uint64(0)
        assert fs.lib().fs_server_submit(srv._h, fs.ctypes.byref(r), fs.ctypes.byref(t)) == fs.FS_E_INVAL


def test_server_enumerate_waits_for_release():
    """Two enumerations that do not fit the budget together: the second is
    materialised only after the first one's rows are released."""
    n, g = 1500, (7, 9, 11, 13)
    c = oracle.count_dp(n, g)
    need = c * len(g) * 2
    with fs.Server(mem_budget_bytes=need + need // 2, max_batch=8) as srv:
        a = srv.submit(fs.REQ_ENUMERATE, n, g)
        b = srv.submit(fs.REQ_ENUMERATE, n, g)
        first = drain(srv, [a])
        assert first[a]["status"] == fs.FS_OK
        time.sleep(0.3)
        assert srv.poll(8, wait_ms=100) == []  # b waits for room
        ra = rows_of(first[a], len(g), 2)
        srv.release(a)
        second = drain(srv, [b])
        check(second[b], fs.REQ_ENUMERATE, n, g)
        assert np.array_equal(rows_of(second[b], len(g), 2), ra)
        srv.release(b)
        with pytest.raises(fs.FsError):
            srv.release(b)


def test_server_serving_workload_full():
    """The serving workload at its full size: 2000 requests drawn like the
    batched ones with n up to 20000 (80 % count, 15 % lengths, 5 % enumerate),
    all submitted at once.  Every count and length range equals the oracle's
    DP; every admitted enumeration's rows sum to n, are strictly increasing in
    the walk order (descending generators) and number |Z|; enumerations larger
    than the 32 GB budget are refused with their exact count."""
    budget = 32 << 30
    reqs = workloads.config5(0, 2000, 1000.0, 20000)
    with fs.Server(mem_budget_bytes=budget, table_bytes=1 << 30, max_batch=512) as srv:
        tickets = {srv.submit(op, n, g, elem_bytes=2): (op, n, g) for (_, op, n, g) in reqs}
        got = {}
        t0 = time.time()
        rng = np.random.default_rng(1)
        while len(got) < len(tickets):
            for r in srv.poll(256, wait_ms=50):
                t = r["ticket"]
                got[t] = r
                op, n, g = tickets[t]
                if op == fs.REQ_ENUMERATE and r["status"] == fs.FS_OK:
                    c, d = r["count"], len(g)
                    if c:
                        # the rows of a random window, checked on the device
                        k = int(min(c, 1 << 20))
                        lo = int(rng.integers(0, c - k + 1))
                        rows = torch.as_tensor(_DevRows(r["rows"] + lo * d * 2, k, d, 2),
                                               device="cuda").to(torch.int64)
                        gv = torch.tensor(g, dtype=torch.int64, device="cuda")
                        assert bool(((rows * gv).sum(1) == n).all()), (n, g)
                        order = sorted(range(d), key=lambda i: -g[i])
                        key = rows[:, order]
                        if k > 1:
                            diff = key[1:] - key[:-1]
                            first = (diff != 0).to(torch.int64).argmax(1)
                            lead = diff.gather(1, first[:, None])[:, 0]
                            assert bool((lead > 0).all()), (n, g)
                    srv.release(t)
            assert time.time() - t0 < 600, f"{len(got)} of {len(tickets)} responses"
    for t, (op, n, g) in tickets.items():
        r = got[t]
        c = oracle.count_dp(n, g)
        assert r["count"] == c, (op, n, g)
        if op == fs.REQ_ENUMERATE and c * len(g) * 2 > budget:
            assert r["status"] == fs.FS_E_CAPACITY
            continue
        assert r["status"] == fs.FS_OK, (op, n, g, r["status"])
        if op in (fs.REQ_LENGTHS, fs.REQ_ENUMERATE) and c > 0:
            assert (r["min_len"], r["max_len"]) == oracle.minmax_dp(n, g), (op, n, g)


def test_server_histogram_work_bound():
    """A histogram whose PAIR walk would visit more than hist_max_leaves leaves is
    refused with FS_E_CAPACITY, its count and length range still exact; one
    under the bound is served with its histogram."""
    big, small = (2000, (11, 13, 17, 19, 23)), (300, (5, 7, 11, 13))
    with fs.Server(mem_budget_bytes=64 << 20, hist_max_leaves=2000) as srv:
        tb = srv.submit(fs.REQ_LENGTHS, *big, hist=True)
        ts = srv.submit(fs.REQ_LENGTHS, *small, hist=True)
        got = drain(srv, [tb, ts])
        r = got[tb]
        assert r["status"] == fs.FS_E_CAPACITY and r["rows"] == 0
        assert r["count"] == oracle.count_dp(*big)
        assert (r["min_len"], r["max_len"]) == oracle.minmax_dp(*big)
        check(got[ts], fs.REQ_LENGTHS, *small, hist=True)
        srv.release(ts)


def test_server_direct_jobs():
    """Count and length requests over the direct-job bound skip the batch and
    run as single-query calls on the job streams (here the bound is one leaf,
    so every such request with more than one leaf does), mixed with batched
    enumerations: every response equals the oracle and the call alone; a
    histogram over the work bound is still refused with its exact count and
    range."""
    reqs = workloads.config5(seed=7, nreq=120, n_max=2500)
    with fs.Server(mem_budget_bytes=512 << 20, max_batch=32, job_streams=3,
                   direct_leaves=1) as srv:
        tickets = {}
        for i, (_, op, n, g) in enumerate(reqs):
            hist = op == fs.REQ_LENGTHS and i % 2 == 0
            tickets[srv.submit(op, n, g, elem_bytes=2, hist=hist)] = (op, n, g, hist)
        got = drain(srv, tickets)
        direct = 0
        for t, (op, n, g, hist) in tickets.items():
            r = got[t]
            check(r, op, n, g, hist=hist)
            direct += r["t_job"] > 0 and r["t_start"] == r["t_job"]
            if op == fs.REQ_ENUMERATE or hist:
                srv.release(t)
        assert direct >= sum(1 for op, _, _, _ in tickets.values() if op != fs.REQ_ENUMERATE) // 2
    big = (2000, (11, 13, 17, 19, 23))
    with fs.Server(mem_budget_bytes=64 << 20, hist_max_leaves=2000, direct_leaves=1) as srv:
        tb = srv.submit(fs.REQ_LENGTHS, *big, hist=True)
        r = drain(srv, [tb])[tb]
        assert r["status"] == fs.FS_E_CAPACITY and r["rows"] == 0 and r["t_start"] == r["t_job"]
        assert r["count"] == oracle.count_dp(*big)
        assert (r["min_len"], r["max_len"]) == oracle.minmax_dp(*big)
    # a histogram larger than the whole budget (858 bins of 8 bytes against 4 KB)
    wide = (6000, (7, 11, 13))
    with fs.Server(mem_budget_bytes=4096, direct_leaves=1) as srv:
        tw = srv.submit(fs.REQ_LENGTHS, *wide, hist=True)
        r = drain(srv, [tw])[tw]
        assert r["status"] == fs.FS_E_CAPACITY and r["rows"] == 0
        assert r["count"] == oracle.count_dp(*wide)
        assert (r["min_len"], r["max_len"]) == oracle.minmax_dp(*wide)


def test_server_long_count_runs_direct():
    """With the default bound, the heavy count query's generators at n = 20000
    (a walk of about 10^7 leaves) run as a job of their own, next to short
    counts that are batched."""
    n, g = workloads.config3(0, n=20000)
    with fs.Server(mem_budget_bytes=64 << 20) as srv:
        tl = srv.submit(fs.REQ_COUNT, n, g)
        ts = srv.submit(fs.REQ_COUNT, 500, (5, 7, 11, 13))
        got = drain(srv, [tl, ts])
        assert got[tl]["status"] == fs.FS_OK and got[tl]["count"] == oracle.count_dp(n, g)
        assert got[tl]["t_start"] == got[tl]["t_job"] > 0
        check(got[ts], fs.REQ_COUNT, 500, (5, 7, 11, 13))
        assert got[ts]["t_job"] == 0.0
