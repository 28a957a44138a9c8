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

