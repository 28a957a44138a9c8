"""The allocation-free count, fs_count_noalloc, called through the C ABI.

It serves callers that cannot let a library allocate device memory (a
framework with its own memory pool or budget, a latency-critical loop that
must not hit cudaMalloc / cudaFree).  Its scratch is a static device array of
FS_NOALLOC_SCRATCH_BYTES, so oversized queries are refused.  This file is
collected last on purpose: a failure here leaves every other test already run.
"""
import ctypes

import pytest

import paper_2405_07989_gb300 as fs
from paper_2405_07989_gb300 import workloads

NOALLOC_BYTES = 4 << 20


def _call(n, gens, dev_ptr, stream):
    g = (ctypes.c_uint32 * len(gens))(*gens)
    return fs.lib().fs_count_noalloc(int(n), g, len(gens), ctypes.c_void_p(dev_ptr),
                                     ctypes.c_void_p(stream))


def test_noalloc_rejects_queries_beyond_the_static_scratch():
    # (d-3)(n+1)*8 bytes of leaf counts: 2 * 1,000,001 * 8 = 16 MB > 4 MiB.
    # The size check comes before any device work, so no GPU is needed.
    st = _call(1_000_000, [97, 89, 83, 79, 73], 16, 0)
    assert st == fs.FS_E_OVERFLOW
    msg = fs.lib().fs_last_error().decode()
    assert "FS_NOALLOC_SCRATCH_BYTES" in msg and str(NOALLOC_BYTES) in msg


@pytest.mark.gpu
def test_noalloc_count_matches_fs_count_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cases = [workloads.CONFIG1, workloads.CONFIG2, (2000, (13, 37, 38, 40, 41, 42)),
             (97, (1, 1, 1)), (17, (5,)), (0, (3, 5, 7)), workloads.config3(0)]
    stream = torch.cuda.current_stream().cuda_stream
    for n, g in cases:
        expect = fs.fs_count(n, g)  # the allocating entry point
        out = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        for k in range(2):
            st = _call(n, list(g), out.data_ptr() + 8 * k, stream)
            assert st == fs.FS_OK, fs.lib().fs_last_error().decode()
        torch.cuda.synchronize()
        assert int(out[0]) == expect and int(out[1]) == expect, (n, g)
