"""The stored full-size oracle results (tests/golden/fullsize_oracle.json,
written by make_golden.py --fullsize from the oracle alone) stay tied to
their inputs: the generators still produce the same pairs, and the stored
figures satisfy the identities that hold for any graph."""
from __future__ import annotations

import hashlib
import json
import os

import pytest

from paper_1907_09575_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize_oracle.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as f:
        return json.load(f)


def test_stored_results_satisfy_identities(gold):
    for name, g in gold.items():
        assert g["per_vertex_sum"] == 3 * g["total"], name       # each triangle has 3 vertices
        assert g["m"] <= g["num_pairs"], name
        assert g["max_outdeg"] <= g["max_deg"] < g["n"], name
        assert g["total"] <= g["wedges_jik"], name                # every triangle is one probe hit


def test_rmat_scale26_pairs_are_the_stored_ones(gold):
    g = gold["rmat-s26"]
    spec = inputs.rmat_graph(1, 26, 16)
    assert (spec.n, spec.num_pairs) == (g["n"], g["num_pairs"])
    src, dst = spec.generate()
    h = hashlib.sha256()
    h.update(src.astype("<i4", copy=False).tobytes())
    h.update(dst.astype("<i4", copy=False).tobytes())
    assert h.hexdigest() == g["pairs_sha256"]


def _digest16(src, dst):
    return hashlib.sha256(src.astype("<i4").tobytes() + dst.astype("<i4").tobytes()).hexdigest()[:16]


def test_stored_batch_results_belong_to_the_batch():
    """tests/golden/batch4096_oracle.json (make_golden.py --batch): one entry
    per graph of the batch, sizes equal to the generator's, pairs digests
    equal for a sample of graphs, and totals within what m edges allow."""
    import math
    with open(os.path.join(os.path.dirname(GOLDEN), "batch4096_oracle.json")) as f:
        b = json.load(f)
    num = b["graphs"]
    assert num == 4096
    for key in ("n", "num_pairs", "m", "total", "pairs_sha256_16"):
        assert len(b[key]) == num, key
    for g in range(num):
        assert b["m"][g] <= b["num_pairs"][g]
        # at most C(k,3) triangles when m >= C(k-1,2): a loose bound from m
        assert b["total"][g] <= b["m"][g] ** 1.5
    for g in list(range(0, num, 97))[:40]:
        spec = inputs.batch_member(b["seed"], g)
        src, dst = spec.generate()
        assert spec.n == b["n"][g] and src.size == b["num_pairs"][g]
        assert _digest16(src, dst) == b["pairs_sha256_16"][g], g
    assert math.isclose(sum(b["m"]), 7.236e8, rel_tol=1e-3)


def test_stored_top_band_requests_belong_to_the_stream():
    """tests/golden/serve_top_oracle.json (make_golden.py --serve-top): the
    first 32 requests of the served stream in the 2^20..2^22-pair band."""
    with open(os.path.join(os.path.dirname(GOLDEN), "serve_top_oracle.json")) as f:
        t = json.load(f)
    lo, hi = t["band"]
    reqs = t["requests"]
    assert len(reqs) == 32 and sum(r["num_pairs"] for r in reqs) > (1 << 26)
    rs = [r["r"] for r in reqs]
    want = [r for r in range(rs[-1] + 1) if inputs.serve_request(t["seed"], r).num_pairs >= lo]
    assert rs == want
    for r in reqs:
        sp = inputs.serve_request(t["seed"], r["r"])
        assert (sp.seed, sp.scale, sp.n, sp.num_pairs) == (r["seed"], r["scale"], r["n"],
                                                           r["num_pairs"])
        assert lo <= r["num_pairs"] <= hi and r["m"] <= r["num_pairs"]
    for r in reqs[:3]:
        src, dst = inputs.serve_request(t["seed"], r["r"]).generate()
        assert _digest16(src, dst) == r["pairs_sha256_16"]


def test_parallel_counter_agrees_with_the_oracle_at_full_size(gold):
    """tests/golden/fullsize_parallel.json (make_golden.py --fullsize-parallel):
    the OpenMP counter in cpu_parallel/, which shares no code with the oracle,
    counted both full-size graphs; every stored figure equals the oracle's."""
    with open(os.path.join(os.path.dirname(GOLDEN), "fullsize_parallel.json")) as f:
        par = json.load(f)
    assert set(par) == set(gold)
    for name, p in par.items():
        for key in ("n", "num_pairs", "total", "per_vertex_sha256", "m", "max_outdeg", "max_deg"):
            assert p[key] == gold[name][key], (name, key)
