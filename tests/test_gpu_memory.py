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
