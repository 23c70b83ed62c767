"""Failure detection without a GPU fault: a bounded device wait made to run
out (a word that nothing publishes) ends, is reported as TC_ETIMEOUT, and
leaves the context usable."""
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


def test_bounded_wait_runs_out_and_reports(tc):
    for limit in (1, 64, 4096):
        assert tc.selftest_wait_timeout(limit) == tc.TC_ETIMEOUT
    assert b"bounded wait" in tc.load().tc_last_error()
    # the context is still usable: a count right after
    spec = inputs.rmat_graph(2, 10, 16)
    s, d = tc.generate_rmat(2, 10, spec.num_pairs)
    g = tc.preprocess(s, d, spec.n)
    assert g.count() > 0
    g.free()
    torch.cuda.synchronize()


def test_selftest_limits(tc):
    assert tc.selftest_wait_timeout(0) == tc.TC_EINVAL
    assert tc.selftest_wait_timeout(1 << 21) == tc.TC_EINVAL
