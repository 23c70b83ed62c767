"""Counting graphs larger than the device budget (tc_graph_offload +
tc_count_tiled): the graph's arrays in host memory, (row block, pivot block)
tiles streamed through device memory -- the single-device form of the
paper's blocked decomposition (Section 5.1, Eq. 4 and Eq. 5).  Every device
byte comes from a caller allocator that refuses to go past the budget, and
the counts equal the oracle's exactly."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1907_09575_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_1907_09575_gb300 import tc as _tc
    _tc.load()
    return _tc


class CappedAllocator:
    """A caller allocator over torch memory that refuses any allocation which
    would take the bytes it has handed out past `cap`."""

    def __init__(self, tc, cap: int):
        self.cap, self.used, self.peak, self.refused = cap, 0, 0, 0
        self.live = {}
        self._alloc = tc.Allocator._fields_[0][1](self.alloc)
        self._free = tc.Allocator._fields_[1][1](self.free)
        self.struct = tc.Allocator(self._alloc, self._free, None)

    def alloc(self, nbytes, ctx, stream):
        nbytes = max(int(nbytes), 1)
        if self.used + nbytes > self.cap:
            self.refused += 1
            return None
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        self.used += nbytes
        self.peak = max(self.peak, self.used)
        return t.data_ptr()

    def free(self, ptr, nbytes, ctx, stream):
        self.live.pop(ptr)
        self.used -= max(int(nbytes), 1)


def offloaded(tc, spec):
    """The graph preprocessed on the device, counted there once (for the
    probes the count kernel makes: tasks whose pivot row is empty are never
    probed), then offloaded."""
    hs, hd = spec.generate()
    g = tc.preprocess(torch.from_numpy(hs).cuda(), torch.from_numpy(hd).cuda(), spec.n, offsets=64)
    st = g.stats()
    st["in_hbm"] = g.count(per_vertex=True)
    st["count_probes"] = sum(g.count_stats()["probes"])
    arena = st["device_bytes"]
    g.offload()
    return g, hs, hd, st, arena


def test_rmat_scale20_within_an_eighth_of_its_arena(tc):
    spec = inputs.rmat_graph(2, 20, 16)
    g, hs, hd, st, arena = offloaded(tc, spec)
    want, want_t = oracle.count(hs, hd, spec.n, per_vertex=True)
    budget = arena // 8
    cap = CappedAllocator(tc, budget)
    total, t, ts = g.count_tiled(budget, per_vertex=True, allocator=cap.struct)
    torch.cuda.synchronize()
    assert total == want and np.array_equal(t, want_t)
    # the in-HBM count of the same graph (its pivots of wide label span take
    # tag tables) equals the oracle too
    hbm_total, hbm_t = st["in_hbm"]
    assert hbm_total == want and np.array_equal(hbm_t.cpu().numpy().astype(np.uint64)[:spec.n], want_t)
    assert cap.refused == 0 and cap.peak <= budget and not cap.live
    assert ts["tiles"] > 4 and ts["row_blocks"] > 1
    assert ts["tile_tasks"] == st["tasks"] and ts["probes"] == st["count_probes"]
    assert g.stats()["device_bytes"] == 0
    # totals only, a quarter of the arena, the library's own pool
    total2, t2, ts2 = g.count_tiled(arena // 4)
    assert total2 == want and t2 is None and ts2["tiles"] <= ts["tiles"]
    g.free()


def test_heavy_pivot_split_over_pivot_blocks(tc):
    """A pivot with more tasks than a pivot block holds: vertex 0 is joined
    to 20,000 leaves and every leaf also to vertex 1 (above 0 in the order),
    so pivot 0 has a task per leaf, each hitting vertex 1; RMAT edges among
    the leaves add structure.  Its tasks are spread over several blocks."""
    leaves = 20000
    n = leaves + 2
    rs, rd = inputs.rmat(7, 14, 200000)
    hs = np.concatenate([np.zeros(leaves, np.int32), np.ones(leaves, np.int32), [0],
                         (rs % leaves + 2).astype(np.int32)]).astype(np.int32)
    hd = np.concatenate([np.arange(2, n, dtype=np.int32), np.arange(2, n, dtype=np.int32), [1],
                         (rd % leaves + 2).astype(np.int32)]).astype(np.int32)
    want, want_t = oracle.count(hs, hd, n, per_vertex=True)
    g = tc.preprocess(torch.from_numpy(hs).cuda(), torch.from_numpy(hd).cuda(), n, offsets=64)
    st = g.stats()
    g.count()
    count_probes = sum(g.count_stats()["probes"])
    g.offload()
    budget = 8 * n + (64 << 10) + (600 << 10)       # a pivot block holds ~12K tasks
    cap = CappedAllocator(tc, budget)
    total, t, ts = g.count_tiled(budget, per_vertex=True, allocator=cap.struct)
    assert total == want and np.array_equal(t, want_t)
    assert cap.refused == 0 and cap.peak <= budget
    assert ts["split_pivots"] >= 1 and ts["tile_tasks"] == st["tasks"]
    assert ts["probes"] == count_probes
    g.free()


def test_large_budget_is_one_tile_per_pivot_block_and_equals_the_device_count(tc):
    spec = inputs.rmat_graph(5, 16, 16)
    hs, hd = spec.generate()
    gd = tc.preprocess(hs, hd, spec.n)
    want, want_t = gd.count(per_vertex=True)
    gd.free()
    g, _, _, st, arena = offloaded(tc, spec)
    total, t, ts = g.count_tiled(64 * arena, per_vertex=True)
    assert total == want and np.array_equal(t, want_t.cpu().numpy().astype(np.uint64))
    assert ts["tiles"] == ts["pivot_blocks"] == ts["row_blocks"] == 1
    g.free()


def test_offloaded_graph_errors(tc):
    spec = inputs.rmat_graph(6, 12, 16)
    g, hs, hd, st, arena = offloaded(tc, spec)
    with pytest.raises(tc.TCError) as ei:          # the device count needs the arena
        g.count()
    assert ei.value.status == tc.TC_EINVAL
    with pytest.raises(tc.TCError) as ei:          # too small for the per-vertex array
        g.count_tiled(8 * spec.n, per_vertex=True)
    assert ei.value.status == tc.TC_ENOMEM
    g.offload()                                    # a second offload does nothing
    assert g.count_tiled(1 << 20)[0] == oracle.count(hs, hd, spec.n)
    gd = tc.preprocess(hs, hd, spec.n)
    with pytest.raises(tc.TCError) as ei:          # not offloaded
        gd.count_tiled(1 << 20)
    assert ei.value.status == tc.TC_EINVAL
    gd.free()
    g.free()
