"""Writes the stored expected values under tests/golden/.

* ``textbook_graphs.json``: small graphs built from their mathematical
  definitions, each with a triangle count (and per-vertex counts where they
  have a closed form) that follows from a cited textbook fact, not from any
  implementation in this repository.
* ``rmat_s14_oracle.json``: the oracle's results on the RMAT scale-14,
  edge-factor-16 graphs of seeds 1, 2, 3 (the small single-graph workload).
* ``fullsize_oracle.json`` (``--fullsize``, tens of minutes and ~30 GB of
  host memory): the oracle's results on the two full-size single-graph
  workloads, RMAT scale 26 (edge factor 16, seed 1) and the Chung-Lu graph
  (5e7 vertices, seed 1): total, a digest of the per-vertex counts, the
  graph statistics.
* ``fullsize_parallel.json`` (``--fullsize-parallel``): the same two graphs
  counted by the OpenMP shared-memory counter in ``cpu_parallel/``, which
  shares no code with the oracle -- a second, independent count at full size.
* ``batch4096_oracle.json`` (``--batch``, a few minutes on all host cores):
  the oracle's total for every one of the 4096 graphs of the batched
  workload (seed 1), with each graph's size and a digest of its pairs.
* ``serve_top_oracle.json`` (``--serve-top``): the oracle's totals for the
  first 32 requests of the served stream (seed 1) whose pair count lies in
  the top band, 2^20..2^22 pairs; together they hold more than 2^26 pairs,
  so a tick carrying all of them takes the large-input deduplication path.
Only ``oracle/`` (``cpu_parallel/`` for ``--fullsize-parallel``) and the
seeded input generators are called.

Run from the repository root:
  python tests/golden/make_golden.py [--fullsize | --fullsize-parallel | --batch | --serve-top]
"""
from __future__ import annotations

import hashlib
import itertools
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def _complete(n):
    return [(a, b) for a in range(n) for b in range(a + 1, n)]


def textbook_graphs():
    out = []

    # Paley graph P(13): x ~ y iff x - y is a nonzero square mod 13.  It is
    # strongly regular with (n, k, lambda, mu) = (13, 6, 2, 3) (Godsil and
    # Royle, Algebraic Graph Theory, Sec. 10.3); each vertex lies in
    # k*lambda/2 = 6 triangles, so there are n*k*lambda/6 = 26.
    q = 13
    sq = {(x * x) % q for x in range(1, q)}
    e = [(a, b) for a in range(q) for b in range(a + 1, q) if (b - a) % q in sq]
    out.append(dict(name="paley13", n=q, edges=e, total=26, per_vertex=[6] * q,
                    source="Paley graph P(13), strongly regular (13,6,2,3): "
                           "t(v) = k*lambda/2, total = n*k*lambda/6"))

    # Kneser graph K(5,2) = Petersen graph: 2-subsets of {0..4}, adjacent iff
    # disjoint.  Girth 5, so no triangles (Godsil and Royle, Sec. 1.6).
    subs = list(itertools.combinations(range(5), 2))
    e = [(a, b) for a in range(len(subs)) for b in range(a + 1, len(subs))
         if not set(subs[a]) & set(subs[b])]
    out.append(dict(name="petersen", n=len(subs), edges=e, total=0,
                    per_vertex=[0] * len(subs), source="Petersen graph K(5,2), girth 5"))

    # Kneser graph K(6,2): a triangle is three pairwise disjoint 2-subsets of
    # a 6-set, i.e. a perfect matching of K_6, of which there are 5!! = 15.
    # Each 2-subset lies in 3!! = 3 of them.
    subs = list(itertools.combinations(range(6), 2))
    e = [(a, b) for a in range(len(subs)) for b in range(a + 1, len(subs))
         if not set(subs[a]) & set(subs[b])]
    out.append(dict(name="kneser6_2", n=len(subs), edges=e, total=15,
                    per_vertex=[3] * len(subs),
                    source="Kneser K(6,2): triangles = perfect matchings of K6 = 5!! = 15"))

    # Octahedron K_{2,2,2}: complement of a perfect matching on 6 vertices;
    # 8 triangular faces, 4 at each vertex, and no other triangles.
    e = [(a, b) for a, b in _complete(6) if b != a + 3]
    out.append(dict(name="octahedron", n=6, edges=e, total=8, per_vertex=[4] * 6,
                    source="octahedron K_{2,2,2}: 8 faces; every triangle is a face"))

    # Rook's graph K_a x K_b (Cartesian product): every triangle lies in one
    # row clique or one column clique: a*C(b,3) + b*C(a,3); vertex t =
    # C(b-1,2) + C(a-1,2).
    a_, b_ = 4, 5
    cells = [(r, c) for r in range(a_) for c in range(b_)]
    e = [(x, y) for x in range(len(cells)) for y in range(x + 1, len(cells))
         if (cells[x][0] == cells[y][0]) != (cells[x][1] == cells[y][1])]
    tv = math.comb(b_ - 1, 2) + math.comb(a_ - 1, 2)
    out.append(dict(name="rook4x5", n=len(cells), edges=e,
                    total=a_ * math.comb(b_, 3) + b_ * math.comb(a_, 3),
                    per_vertex=[tv] * len(cells),
                    source="rook's graph K4 x K5: a*C(b,3) + b*C(a,3)"))

    # Friendship graph F_k: k triangles sharing one vertex (windmill).
    k = 7
    e = []
    for i in range(k):
        e += [(0, 2 * i + 1), (0, 2 * i + 2), (2 * i + 1, 2 * i + 2)]
    out.append(dict(name="friendship7", n=2 * k + 1, edges=e, total=k,
                    per_vertex=[k] + [1] * (2 * k),
                    source="friendship graph F_7: 7 triangles through the centre"))

    # Complete tripartite K_{2,3,4}: a triangle takes one vertex from each
    # part, so 2*3*4 = 24; a vertex of a part of size s lies in
    # (product of the other two part sizes) triangles.
    parts = [2, 3, 4]
    lab = [p for p, s in enumerate(parts) for _ in range(s)]
    e = [(a, b) for a, b in _complete(len(lab)) if lab[a] != lab[b]]
    pv = [24 // parts[p] for p in lab]
    out.append(dict(name="tripartite234", n=len(lab), edges=e, total=24, per_vertex=pv,
                    source="complete tripartite K_{2,3,4}: product of part sizes"))
    return out


def rmat_s14():
    import oracle
    from paper_1907_09575_gb300 import inputs
    res = {}
    for seed in (1, 2, 3):
        spec = inputs.rmat_graph(seed, 14, 16)
        src, dst = spec.generate()
        total, t, st = oracle.count(src, dst, spec.n, per_vertex=True, stats=True)
        res[str(seed)] = dict(
            n=spec.n, num_pairs=spec.num_pairs, total=total,
            per_vertex_sha256=hashlib.sha256(t.astype("<u8").tobytes()).hexdigest(),
            per_vertex_head=[int(x) for x in t[:32]], **st,
            pairs_sha256=hashlib.sha256(src.astype("<i4").tobytes()
                                        + dst.astype("<i4").tobytes()).hexdigest())
    return res


def _record(spec, src, dst):
    import oracle
    total, t, st = oracle.count(src, dst, spec.n, per_vertex=True, stats=True)
    return dict(n=spec.n, num_pairs=int(src.shape[0]), total=total,
                per_vertex_sha256=hashlib.sha256(t.astype("<u8").tobytes()).hexdigest(),
                per_vertex_sum=int(t.sum(dtype="u8")), per_vertex_max=int(t.max()),
                per_vertex_head=[int(x) for x in t[:32]], **st,
                pairs_sha256=hashlib.sha256(src.astype("<i4").tobytes()
                                            + dst.astype("<i4").tobytes()).hexdigest())


def fullsize():
    from paper_1907_09575_gb300 import inputs
    res = {}
    spec = inputs.rmat_graph(1, 26, 16)
    src, dst = spec.generate()
    res["rmat-s26"] = _record(spec, src, dst)
    del src, dst
    spec = inputs.chung_lu_graph(1)
    src, dst = spec.generate()
    res["chunglu"] = _record(spec, src, dst)
    return res


def fullsize_parallel():
    import time
    import cpu_parallel
    from paper_1907_09575_gb300 import inputs
    res = {}
    for name, spec in (("rmat-s26", inputs.rmat_graph(1, 26, 16)), ("chunglu", inputs.chung_lu_graph(1))):
        src, dst = spec.generate()
        t0 = time.perf_counter()
        total, t, st = cpu_parallel.count(src, dst, spec.n, per_vertex=True)
        dt = time.perf_counter() - t0
        res[name] = dict(n=spec.n, num_pairs=int(src.shape[0]), total=total,
                         per_vertex_sha256=hashlib.sha256(t.astype("<u8").tobytes()).hexdigest(),
                         m=st["m"], max_outdeg=st["max_outdeg"], max_deg=st["max_deg"],
                         threads=st["threads"], seconds=round(dt, 1))
        del src, dst, t
    return res


def _pairs_digest(src, dst) -> str:
    return hashlib.sha256(src.astype("<i4").tobytes() + dst.astype("<i4").tobytes()).hexdigest()


def _batch_one(args):
    seed, g = args
    import oracle
    from paper_1907_09575_gb300 import inputs
    spec = inputs.batch_member(seed, g)
    src, dst = spec.generate()
    total, st = oracle.count(src, dst, spec.n, stats=True)
    return g, spec.n, int(src.shape[0]), st["m"], total, _pairs_digest(src, dst)[:16]


def _pool():
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    return ProcessPoolExecutor(max_workers=os.cpu_count() or 1, mp_context=mp.get_context("spawn"))


def batch4096(seed=1, graphs=4096):
    """The oracle over every graph of the batch (one graph per task)."""
    rows = [None] * graphs
    with _pool() as ex:
        for r in ex.map(_batch_one, [(seed, g) for g in range(graphs)], chunksize=8):
            rows[r[0]] = r
    return dict(seed=seed, graphs=graphs,
                n=[r[1] for r in rows], num_pairs=[r[2] for r in rows], m=[r[3] for r in rows],
                total=[r[4] for r in rows], pairs_sha256_16=[r[5] for r in rows],
                source="oracle.count on inputs.batch_member(seed, g), g = 0..graphs-1")


def _serve_one(args):
    seed, r = args
    import oracle
    from paper_1907_09575_gb300 import inputs
    spec = inputs.serve_request(seed, r)
    src, dst = spec.generate()
    total, st = oracle.count(src, dst, spec.n, stats=True)
    return dict(r=r, seed=spec.seed, scale=spec.scale, n=spec.n, num_pairs=spec.num_pairs,
                m=st["m"], total=total, pairs_sha256_16=_pairs_digest(src, dst)[:16])


def serve_top(seed=1, count=32, lo=1 << 20):
    """The first `count` requests of the served stream with >= lo pairs."""
    from paper_1907_09575_gb300 import inputs
    picks, r = [], 0
    while len(picks) < count:
        if inputs.serve_request(seed, r).num_pairs >= lo:
            picks.append(r)
        r += 1
    with _pool() as ex:
        reqs = list(ex.map(_serve_one, [(seed, r) for r in picks]))
    return dict(seed=seed, band=[lo, 1 << 22], requests=reqs,
                source="oracle.count on inputs.serve_request(seed, r) for the listed r")


if __name__ == "__main__":
    for flag, fn, name in (("--fullsize-parallel", fullsize_parallel, "fullsize_parallel.json"),
                           ("--batch", batch4096, "batch4096_oracle.json"),
                           ("--serve-top", serve_top, "serve_top_oracle.json")):
        if flag in sys.argv:
            out = fn()
            with open(os.path.join(HERE, name), "w") as f:
                json.dump(out, f, separators=(",", ":"))
            print("wrote", os.path.join(HERE, name))
            sys.exit(0)
    if "--fullsize" in sys.argv:
        out = fullsize()
        with open(os.path.join(HERE, "fullsize_oracle.json"), "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
        print("wrote", os.path.join(HERE, "fullsize_oracle.json"))
        sys.exit(0)
    with open(os.path.join(HERE, "textbook_graphs.json"), "w") as f:
        json.dump(textbook_graphs(), f, indent=0)
    with open(os.path.join(HERE, "rmat_s14_oracle.json"), "w") as f:
        json.dump(rmat_s14(), f, indent=1, sort_keys=True)
    print("wrote", HERE)
