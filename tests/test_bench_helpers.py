"""Host-side helpers of bench.py: the source hash that keys the recorded DRAM
traffic of the write walk (comments and host-only files do not change it,
code in the kernel's include closure does)."""
import os
import shutil

import pytest

import bench


def test_strip_c_comments_keeps_literals():
    src = ('int a = 1; // note\n/* block\n comment */ const char* s = "x // y /* z */";\n'
           "char q = '\"'; int b;  // end")
    assert bench.strip_c_comments(src) == \
        'int a = 1; const char* s = "x // y /* z */"; char q = \'"\'; int b;'


@pytest.fixture()
def tree(tmp_path, monkeypatch):
    for d in ("include", os.path.join("paper_2405_07989_gb300", "csrc")):
        shutil.copytree(os.path.join(bench.ROOT, d), tmp_path / d)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def _edit(path, old, new):
    s = path.read_text()
    assert old in s
    path.write_text(s.replace(old, new, 1))


def test_kernel_hash_follows_the_include_closure(tree):
    csrc = tree / "paper_2405_07989_gb300" / "csrc"
    h0 = bench.kernel_source_sha("pair_enum")
    # a comment in the kernel's file, a host-only file: same hash
    _edit(csrc / "enum_fixed.cu", "namespace fsi {", "namespace fsi {  // a comment")
    (csrc / "api.cu").write_text((csrc / "api.cu").read_text() + "\nint unrelated_host_symbol;\n")
    assert bench.kernel_source_sha("pair_enum") == h0
    # code in a header the kernel includes: a new hash
    _edit(csrc / "walk.cuh", "namespace fsi {", "namespace fsi {\nconstexpr int probe_constant = 1;")
    assert bench.kernel_source_sha("pair_enum") != h0



def test_recorded_counters_apply_only_to_their_sources(tree, monkeypatch):
    """The recorded traffic and instruction counts are used while the hash of the
    kernel's sources matches, and ignored (None) once the kernel changes."""
    prof = tree / "profiles"
    prof.mkdir()
    sha = bench.kernel_source_sha("pair_count")
    (prof / "count_inst.json").write_text(
        '{"pair_count": {"source_sha": "%s", "alu_warp_inst": 10, "fma_warp_inst": 6,'
        ' "warp_inst": 20, "n": 5, "gens": [1, 2, 3]}}' % sha)
    assert bench.recorded_instructions("pair_count")["warp_inst"] == 20
    _edit(tree / "paper_2405_07989_gb300" / "csrc" / "pair.cu", "namespace fsi {",
          "namespace fsi {\nconstexpr int probe_constant = 2;")
    assert bench.recorded_instructions("pair_count") is None
    assert bench.recorded_instructions("no_such_kernel") is None


class _FakeFs:
    """fs_count over a brute-force count, for the leaf formulas on the host."""

    @staticmethod
    def fs_count(n, gens):
        def rec(i, rest):
            if i == len(gens) - 1:
                return 1 if rest % gens[i] == 0 else 0
            return sum(rec(i + 1, rest - k * gens[i]) for k in range(rest // gens[i] + 1))
        return rec(0, n)


def test_count_roofline_units_are_the_walk_leaves():
    """The PAIR walk visits the prefixes of the first d-2 generators (descending)
    whose residual the last pair's gcd divides; the QUAD walk every prefix of
    the first d-4.  Checked against direct enumeration of those prefixes."""
    import itertools
    import math
    n, g = 60, (12, 10, 9, 7, 6, 4)
    w = sorted(g, reverse=True)
    G = math.gcd(w[-1], w[-2])
    pre = w[:-2]
    direct = 0
    for a in itertools.product(*[range(n // h + 1) for h in pre]):
        phi = sum(x * h for x, h in zip(a, pre))
        if phi <= n and (n - phi) % G == 0:
            direct += 1
    assert bench.visited_leaves(_FakeFs, n, g) == direct
    pre4 = w[:-4]
    direct4 = sum(1 for a in itertools.product(*[range(n // h + 1) for h in pre4])
                  if sum(x * h for x, h in zip(a, pre4)) <= n)
    assert bench.quad_leaves(_FakeFs, n, g) == direct4
    rates = {"add": 1e12}
    r = bench.count_roofline(_FakeFs, n, g, 2.0, rates)
    assert r["leaves_resolved"] == direct and r["frac"] is None
    assert abs(r["useful_frac"] - direct * bench.COUNT_OPS_PER_LEAF / 2e-3 / 1e12) < 1e-12


def test_serving_stages_split_direct_and_batched_requests():
    """The serving breakdown: a batched count (no job), a batched histogram
    (job after the batch), a direct count (its job is its launch) and a request
    never started; every stage non-negative and each request in its stages."""
    def resp(ticket, sub, start, counted, job, done):
        return {"ticket": ticket, "t_submit": sub, "t_start": start, "t_counted": counted,
                "t_job": job, "t_done": done}
    rs = [resp(1, 0.0, 1.0, 3.0, 0.0, 3.5),     # batched, no job
          resp(2, 0.0, 1.0, 3.0, 4.0, 9.0),     # batched, then a job
          resp(3, 0.5, 2.0, 6.0, 2.0, 6.25),    # direct: launched at 2, results at 6
          resp(4, 0.0, 0.0, 0.0, 0.0, 0.1)]     # refused before it ran
    st = bench.serving_stages(rs)
    assert sorted(st["queue"]) == [1.0, 1.0, 1.5]
    assert sorted(st["batch"]) == [2.0, 2.0]
    assert st["direct_job"] == [4.0]
    assert st["job_wait"] == [1.0] and st["job"] == [5.0]
    assert sorted(st["answer"]) == [0.25, 0.5]
    assert all(x >= 0 for v in st.values() for x in v)
