"""Serving: continuously batched requests give exactly their stand-alone
counts, whatever they are batched with; admission respects the HBM budget;
host-side failures (bad specs, over-budget requests, drain timeouts) are
reported as status codes without touching the GPU's state."""
from __future__ import annotations

import json
import os

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


GOLDEN_TOP = os.path.join(os.path.dirname(__file__), "golden", "serve_top_oracle.json")


def test_top_band_requests_in_one_large_tick(tc):
    """The served workload's largest requests (2^20..2^22 pairs), counted in
    one tick whose union holds more than 2^26 pairs -- so preprocessing
    takes the radix-sort deduplication -- mixed with small requests.  Each
    top-band result equals the oracle's total stored for that request by
    tests/golden/make_golden.py --serve-top; each small one its stand-alone
    count."""
    with open(GOLDEN_TOP) as f:
        gold = json.load(f)
    top = gold["requests"]
    for r in top[:4]:                       # the stored specs are the stream's
        sp = inputs.serve_request(gold["seed"], r["r"])
        assert (sp.seed, sp.scale, sp.n, sp.num_pairs) == (r["seed"], r["scale"], r["n"],
                                                           r["num_pairs"])
    small = [small_request(4, r) for r in range(48)]
    order = []
    for k in range(max(len(top), len(small))):
        if k < len(top):
            order.append(("top", top[k]))
        if k < len(small):
            order.append(("small", small[k]))
    specs = [(x["seed"], x["scale"], x["n"], x["num_pairs"]) if kind == "top"
             else (x.seed, x.scale, x.n, x.num_pairs) for kind, x in order]
    srv = tc.Server(hbm_budget_bytes=64 << 30, workers=1, max_batch=256, max_tick_pairs=1 << 28)
    tickets = srv.submit_many(specs)
    srv.drain(timeout_ms=600000)
    res = {r["ticket"]: r for r in srv.poll()}
    srv.free()
    assert len(res) == len(order)
    assert max(r["tick_pairs"] for r in res.values()) > (1 << 26)
    for (kind, x), t in zip(order, tickets):
        r = res[t]
        assert r["status"] == 0
        if kind == "top":
            assert r["triangles"] == x["total"], (x["r"], r["triangles"], x["total"])
        else:
            assert r["triangles"] == standalone(tc, x)


def test_ticks_overlap_and_real_memory_stays_under_the_estimate(tc):
    """With several workers and a backlog, ticks overlap on the device (their
    recorded device spans intersect), and the memory the library's pool
    really hands out stays below the footprint estimate that admission sums
    (64 B per pair + 48 B per vertex), which in turn stays below the budget;
    the estimate is within a factor of 8 of the real high-water mark."""
    dev = torch.cuda.current_device()
    specs = [small_request(6, r, max_log_pairs=18) for r in range(240)]
    budget = 256 << 20
    tc.memory_stats(dev, reset_high=True)
    base = tc.memory_stats(dev)["used"]
    srv = tc.Server(hbm_budget_bytes=budget, workers=3, max_batch=8)
    tickets = srv.submit_many([(x.seed, x.scale, x.n, x.num_pairs) for x in specs])
    srv.drain(timeout_ms=300000)
    res = {r["ticket"]: r for r in srv.poll()}
    st = srv.stats()
    srv.free()
    mem = tc.memory_stats(dev)
    assert len(res) == len(specs) and st["failed"] == 0
    assert st["ticks"] > 3
    assert 0 < st["device_overlap_s"] <= st["device_busy_s"]
    real = mem["used_high"] - base
    assert real <= st["peak_bytes_in_flight"] <= budget, (real, st["peak_bytes_in_flight"])
    assert real * 8 >= st["peak_bytes_in_flight"], (real, st["peak_bytes_in_flight"])
    for x, t in list(zip(specs, tickets))[::24]:
        assert res[t]["triangles"] == standalone(tc, x)
        assert 0 <= res[t]["t_dev_start"] <= res[t]["t_dev_end"]


def test_admission_and_host_side_failures(tc):
    srv = tc.Server(hbm_budget_bytes=1 << 20, workers=1)
    with pytest.raises(tc.TCError) as ei:          # footprint over the whole budget
        srv.submit_rmat(1, 16, 1 << 16, 1 << 16)
    assert ei.value.status == tc.TC_EBUSY
    with pytest.raises(tc.TCError) as ei:          # n beyond 2^scale
        srv.submit_rmat(1, 4, 100, 10)
    assert ei.value.status == tc.TC_EINVAL
    with pytest.raises(tc.TCError) as ei:          # one bad spec: none of the batch is queued
        srv.submit_many([(1, 10, 1000, 2000), (1, 4, 100, 10)])
    assert ei.value.status == tc.TC_EINVAL
    assert srv.stats()["submitted"] == 0
    for r in range(20):
        srv.submit_rmat(r + 1, 10, 1000, 2000)
    lib = tc.load()
    rc = lib.tc_server_drain(srv._h, 0)             # a zero wait with work queued
    assert rc in (tc.TC_OK, tc.TC_ETIMEOUT)
    srv.drain()
    assert srv.stats()["completed"] == 20
    srv.free()
