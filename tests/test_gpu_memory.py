"""The library's device memory pool: freed arenas stay reserved for the next
call, and tc_release_memory hands them back to the device."""
from __future__ import annotations

import pytest

from paper_1907_09575_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_1907_09575_gb300 import tc as _tc
    _tc.load()
    return _tc


def free_bytes() -> int:
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_pool_keeps_and_releases_memory(tc):
    spec = inputs.rmat_graph(3, 21, 16)
    s, d = tc.generate_rmat(3, 21, spec.num_pairs)
    tc.release_memory()
    free0 = free_bytes()
    g = tc.preprocess(s, d, spec.n)
    total = g.count()
    arena = g.stats()["device_bytes"]
    g.free()
    free1 = free_bytes()
    assert arena > 100 << 20
    # the freed arena (and the preprocessing scratch) stayed with the pool
    assert free0 - free1 >= arena // 2
    # a second graph of the same size is served from it
    g = tc.preprocess(s, d, spec.n)
    assert g.count() == total
    g.free()
    free2 = free_bytes()
    assert free1 - free2 < arena // 4
    tc.release_memory(torch.cuda.current_device())
    free3 = free_bytes()
    assert free3 - free2 >= arena // 2
    with pytest.raises(tc.TCError) as ei:
        tc.release_memory(1000)
    assert ei.value.status == tc.TC_EINVAL


class FailingAllocator:
    """A caller allocator over torch memory whose k-th allocation fails."""

    def __init__(self, tc, fail_at: int):
        self.calls = 0
        self.fail_at = fail_at
        self.live = {}
        self._alloc = tc.Allocator._fields_[0][1](self.alloc)
        self._free = tc.Allocator._fields_[1][1](self.free)
        self.struct = tc.Allocator(self._alloc, self._free, None)

    def alloc(self, nbytes, ctx, stream):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr, nbytes, ctx, stream):
        self.live.pop(ptr)


def test_injected_allocation_failures_leak_nothing(tc):
    """Every allocation of preprocessing and counting, failed in turn: the
    call returns TC_ENOMEM and every block it took is given back; when no
    allocation fails the counts are right and freeing the graph returns
    every block."""
    spec = inputs.rmat_graph(4, 12, 16)
    s, d = tc.generate_rmat(4, 12, spec.num_pairs)
    g = tc.preprocess(s, d, spec.n)
    want_total, want_t = g.count(per_vertex=True)
    want_t = want_t.cpu()
    g.free()
    fail_at, completed = 1, False
    while not completed:
        fa = FailingAllocator(tc, fail_at)
        g = None
        try:
            g = tc.preprocess(s, d, spec.n, allocator=fa.struct)
            total, t = g.count(per_vertex=True)
            assert total == want_total and torch.equal(t.cpu(), want_t)
            completed = fa.calls < fail_at          # no allocation failed
        except tc.TCError as e:
            assert e.status == tc.TC_ENOMEM, e
        finally:
            if g is not None:
                g.free()                            # idempotent
        torch.cuda.synchronize()
        assert not fa.live, (fail_at, len(fa.live))
        fail_at += 1
        assert fail_at < 500
    # the library still works with its own pool
    g = tc.preprocess(s, d, spec.n)
    assert g.count() == want_total
    g.free()
