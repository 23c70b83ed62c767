"""Parity at the full workload sizes, in the launch configuration bench.py
times (tc_preprocess + tc_count on device-resident pairs).

The oracle cannot count a billion-edge graph in test time.  Its full
results for these two graphs were computed once, on the host, by
tests/golden/make_golden.py --fullsize (which calls only the oracle and the
seeded generators) and are compared here: total, a digest of every
per-vertex count, and the graph statistics.  The tests also use what the
oracle computes one by one -- the triangles through sampled vertices,
counted from the definition on the host-generated copy of the same pairs --
and properties that hold at any size: the per-vertex counts sum to three
times the total, and relabelling the vertices changes neither the total nor
(up to the relabelling) the per-vertex counts.
"""
from __future__ import annotations

import hashlib
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


def pick_samples(s, d, n, seed):
    """Up to 48 vertices: 36 of modest raw degree, 8 larger, 4 isolated."""
    deg = torch.bincount(s.long(), minlength=n) + torch.bincount(d.long(), minlength=n)
    deg = deg.cpu().numpy()
    rng = np.random.default_rng(seed)
    pick = []
    for lo, hi, k in ((2, 64, 36), (65, 2000, 8), (0, 0, 4)):
        cand = np.flatnonzero((deg >= lo) & (deg <= hi))
        if cand.size:
            pick.extend(rng.choice(cand, size=min(k, cand.size), replace=False).tolist())
    return np.unique(np.asarray(pick, dtype=np.int32))[:64]


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize_oracle.json")


def golden(name):
    if not os.path.exists(GOLDEN):
        return None
    with open(GOLDEN) as f:
        return json.load(f).get(name)


def check_full(tc, s, d, hs, hd, n, offsets, name):
    g = tc.preprocess(s, d, n, offsets=offsets)
    total, t = g.count(per_vertex=True)
    st = g.stats()
    g.free()
    assert int(t.sum().item()) == 3 * total
    gold = golden(name)
    if gold is not None:
        # the oracle's full results on the same graph
        assert total == gold["total"]
        th = t.cpu().numpy().astype("<u8")
        assert hashlib.sha256(th.tobytes()).hexdigest() == gold["per_vertex_sha256"]
        assert st["m"] == gold["m"] and st["max_deg"] == gold["max_deg"]
        assert st["max_outdeg"] == gold["max_outdeg"]
        assert st["probes"] == gold["wedges_jik"] and st["probes_ijk"] == gold["wedges_ijk"]
    samples = pick_samples(s, d, n, seed=n % 9973)
    want = oracle.vertex_triangles(hs, hd, n, samples)
    got = t[torch.from_numpy(samples.astype(np.int64)).cuda()].cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, want)
    assert np.any(want > 0)
    # relabel every vertex by a bijection on [0, n): x -> (x * 0x9E3779B1 + 12345) mod n is a
    # bijection when n is a power of two; for other n use a permutation
    if n & (n - 1) == 0:
        pi = lambda x: (x.long() * 0x9E3779B1 + 12345) % n
    else:
        perm = torch.randperm(n, generator=torch.Generator().manual_seed(7)).cuda()
        pi = lambda x: perm[x.long()]
    s2 = pi(s).int()
    d2 = pi(d).int()
    g2 = tc.preprocess(s2, d2, n, offsets=offsets)
    total2, t2 = g2.count(per_vertex=True)
    g2.free()
    assert total2 == total
    ids = torch.arange(n, device="cuda")
    assert torch.equal(t2[pi(ids)], t)
    return total, st


def test_rmat_scale26_full_size(tc):
    """The RMAT scale-26 workload: 2^30 pairs, int64 offsets, per-vertex."""
    spec = inputs.rmat_graph(1, 26, 16)
    s, d = tc.generate_rmat(1, 26, spec.num_pairs)
    hs, hd = spec.generate()
    # the device copy of the input stream is the host one
    assert np.array_equal(s[-4096:].cpu().numpy(), hs[-4096:])
    total, st = check_full(tc, s, d, hs, hd, spec.n, offsets=64, name="rmat-s26")
    assert st["offset_bytes"] == 8 and st["m"] > 10**9


def test_chung_lu_full_size(tc):
    """The Chung-Lu workload: 5e7 vertices, exponent 2.1, mean degree 40."""
    spec = inputs.chung_lu_graph(1)
    hs, hd = spec.generate()
    s, d = torch.from_numpy(hs).cuda(), torch.from_numpy(hd).cuda()
    total, st = check_full(tc, s, d, hs, hd, spec.n, offsets=64, name="chunglu")
    assert st["max_deg"] > 10**5
