"""The C ABI library loads and exports every entry point include/tc.h declares,
and the binding's struct layouts match the header (checked by compiling a C
probe against the header with gcc).  No compute calls: no GPU needed."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tc.h")


@pytest.fixture(scope="module")
def lib_path():
    from paper_1907_09575_gb300 import build
    try:
        build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    return build.build()


def declared_functions() -> list[str]:
    text = open(HEADER).read()
    return re.findall(r"^TC_API\s+[\w\s\*]+?\b(tc_\w+)\s*\(", text, flags=re.M)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("tc_preprocess", "tc_count", "tc_triangles", "tc_graph_free", "tc_last_error"):
        assert want in names
    from paper_1907_09575_gb300 import tc
    assert sorted(names) == sorted(tc.EXPORTS)


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(declared_functions()) <= exported
    # only the ABI is exported (internal C++ symbols stay hidden)
    assert not [s for s in exported if s.startswith("_ZN2tc")]


def test_binding_loads_without_gpu(lib_path):
    from paper_1907_09575_gb300 import tc
    lib = tc.load(lib_path)
    assert lib.tc_last_error() == b""
    t = tc.tuning_default()
    assert t.small_max_outdeg == 64 and t.slice_max == 4096
    # argument errors are reported without touching the device
    with pytest.raises(tc.TCError) as ei:
        tc._check(lib.tc_count(None, None, None, None, None, None))
    assert ei.value.status == tc.TC_EINVAL
    assert b"NULL" in lib.tc_last_error()


def test_struct_layouts_match_header():
    from paper_1907_09575_gb300 import tc
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "tc.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(tc_tuning), sizeof(tc_graph_stats), sizeof(tc_allocator));
  printf("%zu %zu %zu\n", offsetof(tc_graph_stats, probes), offsetof(tc_graph_stats, device_bytes),
         offsetof(tc_tuning, slice_max));
  printf("%zu %zu %zu %zu\n", sizeof(tc_server_result), offsetof(tc_server_result, tick_pairs),
         sizeof(tc_server_stats), offsetof(tc_server_stats, device_overlap_s));
  printf("%zu %zu %zu %zu %zu\n", sizeof(tc_memory_stats), sizeof(tc_rmat_spec), sizeof(tc_server_config),
         sizeof(tc_triangles_timing), sizeof(tc_tiled_stats));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        a, b, c, e = subprocess.run([exe], capture_output=True, text=True,
                                    check=True).stdout.split("\n")[:4]
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [ctypes.sizeof(tc.Tuning), ctypes.sizeof(tc.GraphStats), ctypes.sizeof(tc.Allocator)]
    assert offs == [tc.GraphStats.probes.offset, tc.GraphStats.device_bytes.offset,
                    tc.Tuning.slice_max.offset]
    assert [int(x) for x in c.split()] == [ctypes.sizeof(tc.ServerResult), tc.ServerResult.tick_pairs.offset,
                                          ctypes.sizeof(tc.ServerStats),
                                          tc.ServerStats.device_overlap_s.offset]
    assert [int(x) for x in e.split()] == [ctypes.sizeof(tc.MemoryStats), ctypes.sizeof(tc.RmatSpec),
                                          ctypes.sizeof(tc.ServerConfig),
                                          ctypes.sizeof(tc.TrianglesTiming),
                                          ctypes.sizeof(tc.TiledStats)]


def test_missing_library_fails_loudly(tmp_path):
    from paper_1907_09575_gb300 import tc
    saved = tc._lib
    tc._lib = None
    try:
        with pytest.raises(RuntimeError, match="missing"):
            tc.load(str(tmp_path / "nope.so"))
    finally:
        tc._lib = saved
