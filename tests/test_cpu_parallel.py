"""The OpenMP shared-memory counter (cpu_parallel/, the speed baseline timed
beside the oracle) against the oracle and closed forms.  It shares no code
with the oracle or the CUDA library, so its agreement with the oracle is an
independent second count."""
from __future__ import annotations

import math

import numpy as np
import pytest

import cpu_parallel
import oracle
from paper_1907_09575_gb300 import inputs


@pytest.mark.parametrize("seed,scale,ef", [(1, 10, 16), (2, 13, 8), (3, 15, 24), (4, 17, 16)])
def test_rmat_against_oracle(seed, scale, ef):
    spec = inputs.rmat_graph(seed, scale, ef)
    s, d = spec.generate()
    want, want_t, st = oracle.count(s, d, spec.n, per_vertex=True, stats=True)
    for threads in (1, 3, 0):
        got, t, pst = cpu_parallel.count(s, d, spec.n, per_vertex=True, threads=threads)
        assert got == want and np.array_equal(t, want_t)
        assert (pst["m"], pst["max_outdeg"], pst["max_deg"]) == (st["m"], st["max_outdeg"],
                                                                 st["max_deg"])


def test_skewed_and_sparse_graphs_against_oracle():
    for spec in (inputs.chung_lu_graph(5, n=200_000, mean_degree=20.0, wmax=5e4),
                 inputs.GraphSpec("gnp", 9, 5000, p=0.004)):
        s, d = spec.generate()
        want, want_t = oracle.count(s, d, spec.n, per_vertex=True)
        got, t, _ = cpu_parallel.count(s, d, spec.n, per_vertex=True)
        assert got == want and np.array_equal(t, want_t)


def test_closed_forms():
    for n in (3, 4, 40, 200):
        e = np.array([(a, b) for a in range(n) for b in range(a + 1, n)], np.int32)
        got, t, _ = cpu_parallel.count(e[:, 0], e[:, 1], n, per_vertex=True)
        assert got == math.comb(n, 3) and np.all(t == math.comb(n - 1, 2))
    # wheel W_n: hub 0 and a rim cycle of n-1 vertices -> n-1 triangles
    n = 12
    rim = list(range(1, n))
    e = [(0, v) for v in rim] + [(rim[i], rim[(i + 1) % len(rim)]) for i in range(len(rim))]
    a = np.array(e, np.int32)
    got, t, _ = cpu_parallel.count(a[:, 1], a[:, 0], n, per_vertex=True)
    assert got == n - 1 and t[0] == n - 1 and np.all(t[1:] == 2)
    # complete bipartite K_{30,40}: no triangles
    a = np.array([(x, 30 + y) for x in range(30) for y in range(40)], np.int32)
    assert cpu_parallel.count(a[:, 0], a[:, 1], 70)[0] == 0


def test_empty_loops_duplicates_and_bad_ids():
    assert cpu_parallel.count([], [], 0)[0] == 0
    assert cpu_parallel.count([0, 1, 1], [0, 1, 1], 2)[0] == 0
    got, t, st = cpu_parallel.count([0, 1, 2, 1, 2, 0, 1], [1, 2, 0, 0, 1, 2, 1], 3, per_vertex=True)
    assert got == 1 and t.tolist() == [1, 1, 1] and st["m"] == 3
    with pytest.raises(ValueError):
        cpu_parallel.count([0, 5], [1, 0], 3)
