"""Serving: continuously batched requests give exactly their stand-alone
counts, whatever they are batched with; admission respects the HBM budget;
host-side failures (bad specs, over-budget requests, drain timeouts) are
reported as status codes without touching the GPU's state."""
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


def small_request(seed, r, max_log_pairs=16):
    """A served request scaled down: pairs log-uniform in 2^10..2^max_log."""
    spec = inputs.serve_request(seed, r)
    rng = np.random.default_rng(seed * 100003 + r)
    m = int(2 ** rng.uniform(10, max_log_pairs))
    e = int(spec.num_pairs and (spec.num_pairs // max(spec.n, 1))) or 8
    n = max(2, -(-m // max(e, 1)))
    scale = max(1, int(np.ceil(np.log2(n))))
    return inputs.GraphSpec("rmat", spec.seed, n, num_pairs=m, scale=scale)


def standalone(tc, spec):
    s, d = tc.generate_rmat(spec.seed, spec.scale, spec.num_pairs, n=spec.n)
    g = tc.preprocess(s, d, spec.n)
    t = g.count()
    g.free()
    return t


def test_served_results_equal_standalone_and_oracle(tc):
    specs = [small_request(1, r) for r in range(160)]
    srv = tc.Server(hbm_budget_bytes=64 << 20, workers=3, max_batch=32)
    tickets = {}
    for k, sp in enumerate(specs):
        tickets[srv.submit_rmat(sp.seed, sp.scale, sp.n, sp.num_pairs)] = k
    srv.drain(timeout_ms=120000)
    res = srv.poll()
    assert len(res) == len(specs)
    st = srv.stats()
    assert st["completed"] == len(specs) and st["failed"] == 0
    assert st["peak_bytes_in_flight"] <= 64 << 20
    assert max(r["tick_requests"] for r in res) > 1          # requests were batched
    for r in res:
        assert r["status"] == 0
        assert r["t_arrival"] <= r["t_admit"] <= r["t_done"]
        sp = specs[tickets[r["ticket"]]]
        assert r["triangles"] == standalone(tc, sp)
    # the oracle on the host-generated copy of a sample
    for r in res[:40]:
        sp = specs[tickets[r["ticket"]]]
        hs, hd = sp.generate()
        assert r["triangles"] == oracle.count(hs, hd, sp.n)
    srv.free()


def test_same_request_alone_and_in_a_mix(tc):
    sp = small_request(2, 7, max_log_pairs=17)
    srv = tc.Server(workers=2)
    srv.submit_rmat(sp.seed, sp.scale, sp.n, sp.num_pairs)
    srv.drain()
    alone = srv.poll()
    assert len(alone) == 1 and alone[0]["tick_requests"] == 1
    mix = [small_request(3, r) for r in range(60)]
    want = None
    for k, m in enumerate(mix):
        if k == 30:
            want = srv.submit_rmat(sp.seed, sp.scale, sp.n, sp.num_pairs)
        srv.submit_rmat(m.seed, m.scale, m.n, m.num_pairs)
    srv.drain()
    res = {r["ticket"]: r for r in srv.poll()}
    assert res[want]["triangles"] == alone[0]["triangles"] == standalone(tc, sp)
    srv.free()


def test_admission_and_host_side_failures(tc):
    srv = tc.Server(hbm_budget_bytes=1 << 20, workers=1)
    with pytest.raises(tc.TCError) as ei:          # footprint over the whole budget
        srv.submit_rmat(1, 16, 1 << 16, 1 << 16)
    assert ei.value.status == tc.TC_EBUSY
    with pytest.raises(tc.TCError) as ei:          # n beyond 2^scale
        srv.submit_rmat(1, 4, 100, 10)
    assert ei.value.status == tc.TC_EINVAL
    for r in range(20):
        srv.submit_rmat(r + 1, 10, 1000, 2000)
    lib = tc.load()
    rc = lib.tc_server_drain(srv._h, 0)             # a zero wait with work queued
    assert rc in (tc.TC_OK, tc.TC_ETIMEOUT)
    srv.drain()
    assert srv.stats()["completed"] == 20
    srv.free()
