"""The allocation-free count, fs_count_noalloc, called through the C ABI.

It serves callers that cannot let a library allocate device memory (a
framework with its own memory pool or budget, a latency-critical loop that
must not hit cudaMalloc / cudaFree).  Its scratch is a static device array of
FS_NOALLOC_SCRATCH_BYTES, so oversized queries are refused.  The library
counts its own allocations (fs_alloc_counts), so the tests check that the
calls add none, also in a fresh process where no allocating call came first.
This file is collected last on purpose: a failure here leaves every other
test already run.
"""
import ctypes
import json
import os
import subprocess
import sys

import pytest

import paper_2405_07989_gb300 as fs
from paper_2405_07989_gb300 import workloads

NOALLOC_BYTES = 4 << 20
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _call(n, gens, dev_ptr, stream):
    g = (ctypes.c_uint32 * len(gens))(*gens)
    return fs.lib().fs_count_noalloc(int(n), g, len(gens), ctypes.c_void_p(dev_ptr),
                                     ctypes.c_void_p(stream))


def test_noalloc_rejects_queries_beyond_the_static_scratch():
    # (d-3)(n+1)*8 bytes of leaf counts: 2 * 1,000,001 * 8 = 16 MB > 4 MiB.
    # The size check comes before any device work, so no GPU is needed.
    before = fs.fs_alloc_counts()
    st = _call(1_000_000, [97, 89, 83, 79, 73], 16, 0)
    assert st == fs.FS_E_OVERFLOW
    msg = fs.lib().fs_last_error().decode()
    assert "FS_NOALLOC_SCRATCH_BYTES" in msg and str(NOALLOC_BYTES) in msg
    assert fs.fs_alloc_counts() == before


CASES = [workloads.CONFIG1, workloads.CONFIG2, (2000, (13, 37, 38, 40, 41, 42)),
         (97, (1, 1, 1)), (17, (5,)), (0, (3, 5, 7)), workloads.config3(0)]


@pytest.mark.gpu
def test_noalloc_count_matches_fs_count_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stream = torch.cuda.current_stream().cuda_stream
    for n, g in CASES:
        expect = fs.fs_count(n, g)  # the allocating entry point
        out = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        before = fs.fs_alloc_counts()
        for k in range(2):
            st = _call(n, list(g), out.data_ptr() + 8 * k, stream)
            assert st == fs.FS_OK, fs.lib().fs_last_error().decode()
        torch.cuda.synchronize()
        assert fs.fs_alloc_counts() == before, (n, g)  # the calls allocated nothing
        assert int(out[0]) == expect and int(out[1]) == expect, (n, g)


# Run in a child process: the allocation-free calls come first, before any
# allocating call of the library, and must leave its allocation counts at zero;
# fs_count then gives the values to compare with.
_CHILD = r"""
import ctypes, json, sys
import torch
import paper_2405_07989_gb300 as fs
cases = json.loads(sys.argv[1])
torch.cuda.set_device(0)
stream = torch.cuda.current_stream().cuda_stream
out = torch.full((2 * len(cases),), -1, dtype=torch.int64, device="cuda")
torch.cuda.synchronize()
status = []
for i, (n, g) in enumerate(cases):
    arr = (ctypes.c_uint32 * len(g))(*g)
    for k in range(2):
        status.append(fs.lib().fs_count_noalloc(n, arr, len(g),
                      ctypes.c_void_p(out.data_ptr() + 8 * (2 * i + k)), ctypes.c_void_p(stream)))
torch.cuda.synchronize()
allocs = fs.fs_alloc_counts()
got = [int(x) for x in out.tolist()]
expect = [fs.fs_count(n, g) for n, g in cases]
print(json.dumps({"status": status, "allocs": list(allocs), "got": got, "expect": expect}))
"""


@pytest.mark.gpu
def test_noalloc_first_in_a_fresh_process_allocates_nothing():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cases = [[n, list(g)] for n, g in CASES]
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", _CHILD, json.dumps(cases)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["status"] == [fs.FS_OK] * (2 * len(cases))
    assert res["allocs"] == [0, 0]
    for i, e in enumerate(res["expect"]):
        assert res["got"][2 * i] == e and res["got"][2 * i + 1] == e, cases[i]
