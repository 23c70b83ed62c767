"""The allocation-free entry point tc_triangles_static, called through the C ABI.

It serves callers that cannot allocate device memory when they need a count
(all memory already handed to another allocator, or steady-state loops that
must not allocate): every buffer comes from the library's fixed static
scratch.  Its results must equal those of the allocating path
(tc_preprocess + tc_count) exactly -- counts are integers, the tolerance our
tests use is zero -- on two calls in a row, the second reusing the scratch
the first left behind.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1907_09575_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_1907_09575_gb300 import tc as _tc
    _tc.load()
    return _tc


def allocating_path(tc, s, d, n):
    g = tc.preprocess(s, d, n)
    total, pv = g.count(per_vertex=True)
    g.free()
    return total, pv.cpu().numpy()


def static_path(tc, s, d, n):
    lib = tc.load()
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    pv = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.tc_triangles_static(s.data_ptr(), d.data_ptr(), int(s.shape[0]), n,
                                 total.data_ptr(), pv.data_ptr(), st)
    assert rc == tc.TC_OK, lib.tc_last_error()
    torch.cuda.synchronize()
    return int(total.item()), pv[:n].cpu().numpy()


def test_static_entry_matches_allocating_path_twice(tc):
    # call 1: the small RMAT workload (scale 14, edge factor 16) = the limit
    # on pairs; call 2: a different graph on the same scratch
    spec1 = inputs.rmat_graph(1, 14, 16)
    assert spec1.num_pairs == tc.TC_STATIC_MAX_PAIRS
    s1, d1 = tc.generate_rmat(1, 14, spec1.num_pairs)
    spec2 = inputs.GraphSpec("gnp", 7, 3000, p=0.01)
    h2s, h2d = spec2.generate()
    s2, d2 = torch.from_numpy(h2s).cuda(), torch.from_numpy(h2d).cuda()
    for (s, d, n) in ((s1, d1, spec1.n), (s2, d2, spec2.n)):
        want_total, want_pv = allocating_path(tc, s, d, n)
        got_total, got_pv = static_path(tc, s, d, n)
        assert got_total == want_total
        assert np.array_equal(got_pv, want_pv)
    # and once more on the first graph after the second overwrote the scratch
    assert static_path(tc, s1, d1, spec1.n)[0] == allocating_path(tc, s1, d1, spec1.n)[0]


def test_static_entry_rejects_sizes_beyond_its_limits(tc):
    lib = tc.load()
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    big = torch.zeros(tc.TC_STATIC_MAX_PAIRS + 1, dtype=torch.int32, device="cuda")
    rc = lib.tc_triangles_static(big.data_ptr(), big.data_ptr(), big.shape[0], 10,
                                 total.data_ptr(), None, None)
    assert rc == tc.TC_EINVAL
    assert b"static limits" in lib.tc_last_error()
    rc = lib.tc_triangles_static(big.data_ptr(), big.data_ptr(), 10,
                                 tc.TC_STATIC_MAX_VERTICES + 1, total.data_ptr(), None, None)
    assert rc == tc.TC_EINVAL
    # the binding's wrapper gives the same total as the C call
    s, d = tc.generate_rmat(3, 12, 16 << 12)
    assert tc.triangles_static(s, d, 1 << 12) == allocating_path(tc, s, d, 1 << 12)[0]


def unique_pairs(seed, scale, count):
    """Exactly `count` distinct undirected pairs (no self-loops) on 2^scale
    vertices, in the order an RMAT stream first produces them."""
    n = 1 << scale
    s, d = inputs.rmat(seed, scale, 4 * count)
    lo, hi = np.minimum(s, d).astype(np.int64), np.maximum(s, d).astype(np.int64)
    keep = lo != hi
    key = (lo << 32 | hi)[keep]
    _, first = np.unique(key, return_index=True)
    first = np.sort(first)[:count]
    assert first.size == count
    return s[keep][first].copy(), d[keep][first].copy(), n


def test_static_entry_at_its_documented_limits(tc):
    """The worst case the scratch is sized for: TC_STATIC_MAX_VERTICES
    vertices, TC_STATIC_MAX_PAIRS pairs that are all distinct edges (so every
    temporary is at its largest), per-vertex counts requested."""
    import oracle
    hs, hd, n = unique_pairs(11, 16, tc.TC_STATIC_MAX_PAIRS)
    assert n == tc.TC_STATIC_MAX_VERTICES and hs.size == tc.TC_STATIC_MAX_PAIRS
    s, d = torch.from_numpy(hs).cuda(), torch.from_numpy(hd).cuda()
    want_total, want_pv = allocating_path(tc, s, d, n)
    got_total, got_pv = static_path(tc, s, d, n)       # asserts TC_OK, not TC_ENOMEM
    assert got_total == want_total == oracle.count(hs, hd, n)
    assert np.array_equal(got_pv, want_pv)


def test_static_entry_leaves_device_memory_untouched(tc):
    """A call on pre-allocated inputs and outputs changes the device's free
    memory by nothing: no allocation by the library, its pool or the runtime."""
    lib = tc.load()
    dev = torch.cuda.current_device()
    s, d = tc.generate_rmat(5, 14, 1 << 17)
    n = 1 << 14
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    pv = torch.zeros(n, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    # first call: loads the kernels and looks up the scratch address
    assert lib.tc_triangles_static(s.data_ptr(), d.data_ptr(), s.shape[0], n, total.data_ptr(),
                                   pv.data_ptr(), st) == tc.TC_OK
    torch.cuda.synchronize()
    first = int(total.item())
    tc.release_memory(dev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(2):
        assert lib.tc_triangles_static(s.data_ptr(), d.data_ptr(), s.shape[0], n,
                                       total.data_ptr(), pv.data_ptr(), st) == tc.TC_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert int(total.item()) == first
