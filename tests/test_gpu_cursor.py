"""The resumable cursor and the streamed host enumerate: every window of rows
equals the same rows of the whole ordered enumerate (byte for byte), seeking
resumes anywhere, and the host variant equals the device buffer."""
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


def whole(n, g, cfg=None, elem_bytes=4):
    c = fs.fs_count(n, g)
    dt = torch.int16 if elem_bytes == 2 else torch.int32
    out = torch.empty((max(c, 1), len(g)), dtype=dt, device="cuda")
    fs.fs_enumerate(n, g, out, cap=c, elem_bytes=elem_bytes, cfg=cfg)
    return out[:c].cpu()


CASES = [workloads.CONFIG1, (700, (5, 7, 9, 11, 13)), (1200, (11, 13, 17, 19, 23, 29)),
         (300, (3, 5)), (97, (7,)), (40, (41, 43, 47)), (0, (3, 5, 7))]


@pytest.mark.parametrize("keep", [False, True])
@pytest.mark.parametrize("elem_bytes", [4, 2])
def test_cursor_windows_concatenate_to_the_whole(keep, elem_bytes):
    cfg = fs.make_config(keep_order=keep)
    dt = torch.int16 if elem_bytes == 2 else torch.int32
    for n, g in CASES:
        ref = whole(n, g, cfg, elem_bytes)
        total = ref.shape[0]
        assert total == oracle.count_dp(n, g)
        for cap in (1, 7, 1000, 4099, max(total, 1)):
            with fs.Cursor(n, g, elem_bytes, cfg) as cur:
                assert cur.count() == total
                buf = torch.full((cap, len(g)), -3, dtype=dt, device="cuda")

                def windows(limit):
                    parts = []
                    while len(parts) < limit:
                        buf.fill_(-3)
                        m = cur.next(buf, cap)
                        if m == 0:
                            break
                        parts.append(buf[:m].cpu().clone())
                        if m < cap:
                            assert torch.all(buf[m:].cpu() == -3)  # nothing past the window
                    return torch.cat(parts) if parts else ref[:0]

                # the first 40 windows, then (small windows on a large set)
                # the last 40 after a seek
                head = windows(40)
                assert torch.equal(head, ref[:head.shape[0]]), (n, g, cap)
                if cur.tell() < total:
                    start = max(cur.tell(), total - 40 * cap)
                    cur.seek(start)
                    tail = windows(10**9)
                    assert torch.equal(tail, ref[start:]), (n, g, cap)
                assert cur.tell() == total


def test_cursor_seek_resumes_anywhere():
    n, g = 1500, (11, 13, 17, 19, 23)
    ref = whole(n, g)
    total = ref.shape[0]
    rng = np.random.default_rng(4)
    buf = torch.empty((5000, len(g)), dtype=torch.int32, device="cuda")
    with fs.Cursor(n, g) as cur:
        for pos in list(rng.integers(0, total, 20)) + [0, total - 1, total]:
            cap = int(rng.integers(1, 5000))
            cur.seek(int(pos))
            m = cur.next(buf, cap)
            assert m == min(cap, total - int(pos))
            assert torch.equal(buf[:m].cpu(), ref[int(pos):int(pos) + m])
            assert cur.tell() == int(pos) + m
        with pytest.raises(fs.FsError):
            cur.seek(total + 1)


def test_cursor_rows_are_the_oracles_set():
    n, g = workloads.CONFIG1
    with fs.Cursor(n, g, cfg=fs.make_config(keep_order=True)) as cur:
        buf = torch.empty((cur.count(), len(g)), dtype=torch.int32, device="cuda")
        assert cur.next(buf) == cur.count()
    assert np.array_equal(buf.cpu().numpy(), oracle.enumerate_sorted(n, g))


def test_cursor_refuses_other_methods():
    for m in (fs.METHOD_PLAIN, fs.METHOD_TRIPLE, fs.METHOD_QUAD):
        with pytest.raises(fs.FsError) as e:
            fs.Cursor(500, (5, 7, 11, 13, 17), cfg=fs.make_config(method=m))
        assert e.value.status == fs.FS_E_NOTIMPL


@pytest.mark.parametrize("pinned", [True, False])
def test_enumerate_host_equals_device(pinned):
    for n, g in CASES + [(2000, (11, 13, 17, 19, 23, 29))]:
        ref = whole(n, g)
        c = ref.shape[0]
        host = torch.full((max(c, 1), len(g)), -1, dtype=torch.int32, pin_memory=pinned)
        assert fs.fs_enumerate_host(n, g, host, cap=c) == c
        assert torch.equal(host[:c], ref), (n, g)
    # capacity: the first cap rows, FS_E_CAPACITY with the count
    n, g = 700, (5, 7, 9, 11, 13)
    ref = whole(n, g)
    host = torch.full((100, 5), -1, dtype=torch.int32, pin_memory=pinned)
    with pytest.raises(fs.FsError) as e:
        fs.fs_enumerate_host(n, g, host, cap=60)
    assert e.value.status == fs.FS_E_CAPACITY
    assert fs.fs_enumerate_host(n, g, host, cap=60, allow_capacity=True) == ref.shape[0]
    assert torch.equal(host[:60], ref[:60]) and torch.all(host[60:] == -1)


def test_enumerate_host_config2_full():
    """72,082,790 rows streamed to pinned host memory through 128 MB windows
    equal the device enumerate byte for byte."""
    n, g = workloads.CONFIG2
    c = fs.fs_count(n, g)
    dev = torch.empty((c, len(g)), dtype=torch.int32, device="cuda")
    assert fs.fs_enumerate(n, g, dev) == c
    host = torch.empty((c, len(g)), dtype=torch.int32, pin_memory=True)
    assert fs.fs_enumerate_host(n, g, host) == c
    assert torch.equal(host, dev.cpu())
    del dev, host
    torch.cuda.empty_cache()
