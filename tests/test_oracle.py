"""Pins for the CPU oracle: it is checked against things other than itself.

* brute force over all vertex triples (n <= 40);
* dense trace(A^3)/6 and diag(A^3)/2 in int64 linear algebra (n <= 600);
* closed forms: K_n, wheels, cycles, stars, trees, bipartite graphs;
* textbook graphs with known counts (tests/golden/textbook_graphs.json);
* invariants: sum of per-vertex counts = 3 x total, vertex relabelling,
  duplicated / reversed pairs and self-loops, disjoint unions, isolated
  vertices;
* networkx's ``triangles`` where networkx is installed;
* mutation tests: oracle builds with a planted mistake must fail a pin.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1907_09575_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def as_arrays(edges):
    if len(edges) == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    e = np.asarray(edges, dtype=np.int64)
    return e[:, 0].astype(np.int32), e[:, 1].astype(np.int32)


def brute_force(n, edges):
    adj = np.zeros((n, n), dtype=bool)
    for a, b in edges:
        if a != b:
            adj[a, b] = adj[b, a] = True
    total, t = 0, np.zeros(n, dtype=np.int64)
    for a, b, c in itertools.combinations(range(n), 3):
        if adj[a, b] and adj[a, c] and adj[b, c]:
            total += 1
            t[a] += 1
            t[b] += 1
            t[c] += 1
    return total, t


def trace_a3(n, edges):
    A = np.zeros((n, n), dtype=np.int64)
    for a, b in edges:
        if a != b:
            A[a, b] = A[b, a] = 1
    A3 = A @ A @ A
    d = np.diag(A3)
    assert d.sum() % 6 == 0 and np.all(d % 2 == 0)
    return int(d.sum() // 6), d // 2


def random_pairs(rng, n, m, loops=True, dups=True):
    src = rng.integers(0, n, size=m)
    dst = rng.integers(0, n, size=m)
    if not loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    e = list(zip(src.tolist(), dst.tolist()))
    if dups and e:
        e += [(b, a) for a, b in e[: len(e) // 3]]
    return e


# ----------------------------------------------------------------------------
# brute force and linear algebra
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(60))
def test_matches_triple_loop(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    m = int(rng.integers(0, n * n // 2 + 2))
    e = random_pairs(rng, n, m)
    s, d = as_arrays(e)
    total, t = oracle.count(s, d, n, per_vertex=True)
    bt, bv = brute_force(n, e)
    assert total == bt
    assert np.array_equal(t.astype(np.int64), bv)


@pytest.mark.parametrize("seed", range(12))
def test_matches_trace_a3_random(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(50, 600))
    p = float(rng.uniform(0.01, 0.3))
    m = int(p * n * n / 2)
    e = random_pairs(rng, n, m)
    s, d = as_arrays(e)
    total, t = oracle.count(s, d, n, per_vertex=True)
    tt, tv = trace_a3(n, e)
    assert total == tt
    assert np.array_equal(t.astype(np.int64), tv)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_matches_trace_a3_rmat(seed):
    # skewed RMAT degree profile, scale 9 (512 vertices), edge factor 16
    spec = inputs.rmat_graph(seed, 9, 16)
    s, d = spec.generate()
    total, t = oracle.count(s, d, spec.n, per_vertex=True)
    tt, tv = trace_a3(spec.n, list(zip(s.tolist(), d.tolist())))
    assert total == tt
    assert np.array_equal(t.astype(np.int64), tv)


# ----------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 10, 33, 64])
def test_complete_graph(n):
    e = [(a, b) for a in range(n) for b in range(a + 1, n)]
    s, d = as_arrays(e)
    total, t = oracle.count(s, d, n, per_vertex=True)
    assert total == math.comb(n, 3)
    assert np.all(t == math.comb(n - 1, 2)) if n else t.size == 0


@pytest.mark.parametrize("n", [4, 5, 6, 9, 50, 301])
def test_wheel(n):
    # W_n: hub 0 plus a rim cycle on n-1 vertices; n-1 triangles for n >= 5,
    # and W_4 = K_4 has 4.
    rim = list(range(1, n))
    e = [(0, r) for r in rim] + [(rim[i], rim[(i + 1) % len(rim)]) for i in range(len(rim))]
    s, d = as_arrays(e)
    total, t = oracle.count(s, d, n, per_vertex=True)
    if n == 4:
        assert total == 4 and np.all(t == 3)
    else:
        assert total == n - 1
        assert t[0] == n - 1 and np.all(t[1:] == 2)


@pytest.mark.parametrize("n", [3, 4, 5, 8, 101])
def test_cycle(n):
    e = [(i, (i + 1) % n) for i in range(n)]
    s, d = as_arrays(e)
    assert oracle.count(s, d, n) == (1 if n == 3 else 0)


@pytest.mark.parametrize("seed", range(6))
def test_bipartite_and_trees_have_none(seed):
    rng = np.random.default_rng(seed)
    a, b = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    e = [(x, a + y) for x in range(a) for y in range(b) if rng.random() < 0.5]
    s, d = as_arrays(e)
    assert oracle.count(s, d, a + b) == 0
    # random tree (Pruefer-free: attach each vertex to an earlier one)
    n = int(rng.integers(2, 200))
    e = [(v, int(rng.integers(0, v))) for v in range(1, n)]
    s, d = as_arrays(e)
    assert oracle.count(s, d, n) == 0
    # star
    e = [(0, v) for v in range(1, n)]
    s, d = as_arrays(e)
    assert oracle.count(s, d, n) == 0


def test_textbook_graphs():
    with open(os.path.join(GOLDEN, "textbook_graphs.json")) as f:
        graphs = json.load(f)
    assert len(graphs) >= 6
    for g in graphs:
        s, d = as_arrays(g["edges"])
        total, t = oracle.count(s, d, g["n"], per_vertex=True)
        assert total == g["total"], g["name"]
        assert t.tolist() == g["per_vertex"], g["name"]


# ----------------------------------------------------------------------------
# invariants
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_invariants(seed):
    rng = np.random.default_rng(500 + seed)
    spec = inputs.rmat_graph(seed + 1, 10, 8)
    s, d = spec.generate()
    n = spec.n
    total, t = oracle.count(s, d, n, per_vertex=True)
    assert int(t.sum()) == 3 * total

    # vertex relabelling
    pi = rng.permutation(n).astype(np.int32)
    t2, v2 = oracle.count(pi[s], pi[d], n, per_vertex=True)
    assert t2 == total and np.array_equal(v2[pi], t)

    # duplicated and reversed pairs, self-loops, shuffled order
    extra = rng.integers(0, s.size, size=s.size // 2)
    loops = rng.integers(0, n, size=100).astype(np.int32)
    s3 = np.concatenate([s, d[extra], loops, s[extra]])
    d3 = np.concatenate([d, s[extra], loops, d[extra]])
    order = rng.permutation(s3.size)
    assert oracle.count(s3[order], d3[order], n) == total

    # disjoint union adds; isolated vertices change nothing
    spec2 = inputs.rmat_graph(seed + 100, 9, 8)
    sb, db = spec2.generate()
    tb = oracle.count(sb, db, spec2.n)
    su = np.concatenate([s, sb + n]).astype(np.int32)
    du = np.concatenate([d, db + n]).astype(np.int32)
    assert oracle.count(su, du, n + spec2.n + 17) == total + tb


def test_networkx_agrees():
    nx = pytest.importorskip("networkx")
    for seed in range(5):
        spec = inputs.rmat_graph(seed + 7, 11, 12)
        s, d = spec.generate()
        G = nx.Graph()
        G.add_nodes_from(range(spec.n))
        G.add_edges_from((int(a), int(b)) for a, b in zip(s, d) if a != b)
        tri = nx.triangles(G)
        total, t = oracle.count(s, d, spec.n, per_vertex=True)
        assert total == sum(tri.values()) // 3
        assert all(int(t[v]) == tri[v] for v in range(spec.n))


def test_stats_against_definitions():
    spec = inputs.rmat_graph(3, 10, 16)
    s, d = spec.generate()
    _, st = oracle.count(s, d, spec.n, stats=True)
    a = np.minimum(s, d).astype(np.int64)
    b = np.maximum(s, d).astype(np.int64)
    keep = a != b
    keys = np.unique(a[keep] * spec.n + b[keep])
    assert st["m"] == keys.size
    deg = np.bincount(keys // spec.n, minlength=spec.n) + np.bincount(keys % spec.n, minlength=spec.n)
    assert st["max_deg"] == deg.max()


def test_invalid_input_rejected():
    with pytest.raises(ValueError):
        oracle.count([0, 5], [1, 2], 5)
    with pytest.raises(ValueError):
        oracle.count([-1], [1], 5)


# ----------------------------------------------------------------------------
# per-vertex counting from the definition (for sampled checks on big graphs)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_vertex_triangles_matches(seed):
    rng = np.random.default_rng(seed)
    spec = inputs.rmat_graph(seed + 20, 11, 16)
    s, d = spec.generate()
    _, t = oracle.count(s, d, spec.n, per_vertex=True)
    samples = rng.choice(spec.n, size=40, replace=False).astype(np.int32)
    samples[0] = int(np.argmax(t))
    got = oracle.vertex_triangles(s, d, spec.n, samples)
    assert np.array_equal(got, t[samples])
    # and against brute force on a tiny graph
    e = random_pairs(rng, 30, 200)
    s2, d2 = as_arrays(e)
    _, bv = brute_force(30, e)
    got = oracle.vertex_triangles(s2, d2, 30, np.arange(30, dtype=np.int32))
    assert np.array_equal(got.astype(np.int64), bv)


def test_golden_rmat_s14_stable():
    """The stored oracle results for the small RMAT workload still hold
    (guards the generator and the oracle against silent drift)."""
    import hashlib
    with open(os.path.join(GOLDEN, "rmat_s14_oracle.json")) as f:
        gold = json.load(f)
    for seed, g in gold.items():
        spec = inputs.rmat_graph(int(seed), 14, 16)
        s, d = spec.generate()
        h = hashlib.sha256(s.astype("<i4").tobytes() + d.astype("<i4").tobytes()).hexdigest()
        assert h == g["pairs_sha256"]
        total, t = oracle.count(s, d, spec.n, per_vertex=True)
        assert total == g["total"]
        assert hashlib.sha256(t.astype("<u8").tobytes()).hexdigest() == g["per_vertex_sha256"]


# ----------------------------------------------------------------------------
# mutation tests: each planted mistake is caught by at least one pin
# ----------------------------------------------------------------------------

def _pins_pass(mutant: int) -> bool:
    def cnt(e, n, pv=False):
        s, d = as_arrays(e)
        return oracle.count(s, d, n, per_vertex=pv, mutant=mutant)
    try:
        # closed forms
        for n in (4, 6, 9):
            tot, t = cnt(_kn(n), n, True)
            if tot != math.comb(n, 3) or int(t.sum()) != 3 * tot:
                return False
        # brute force with self-loops and duplicates in the input
        rng = np.random.default_rng(7)
        for _ in range(20):
            n = int(rng.integers(3, 25))
            e = random_pairs(rng, n, int(rng.integers(n, n * n)))
            tot, t = cnt(e, n, True)
            bt, bv = brute_force(n, e)
            if tot != bt or not np.array_equal(t.astype(np.int64), bv):
                return False
    except (ValueError, OSError):
        return False
    return True


def _kn(n):
    return [(a, b) for a in range(n) for b in range(a + 1, n)]


def test_pins_pass_on_the_oracle():
    assert _pins_pass(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6])
def test_planted_mistake_is_caught(mutant):
    assert not _pins_pass(mutant)
