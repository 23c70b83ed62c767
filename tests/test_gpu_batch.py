"""Batched counting (one persistent launch over many graphs) against the
oracle and against counting each graph alone.  Counts are integers: exact."""
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


def small_batch(seed, count, max_log_n=12):
    """Uneven graphs shaped like the 4096-graph batch, scaled down."""
    rng = np.random.default_rng(seed)
    specs = []
    for g in range(count):
        n = int(2 ** rng.uniform(4, max_log_n))
        d = float(rng.uniform(2, 40))
        if g % 2 == 0:
            specs.append(inputs.GraphSpec("gnp", seed * 1000 + g, max(n, 2), p=min(1.0, d / max(n - 1, 1))))
        else:
            scale = max(1, int(np.ceil(np.log2(max(n, 2)))))
            specs.append(inputs.GraphSpec("rmat", seed * 1000 + g, max(n, 2),
                                          num_pairs=int(n * d / 2), scale=scale))
    return specs


def build(tc, specs, offsets=None):
    graphs, want = [], []
    for k, sp in enumerate(specs):
        s, d = sp.generate()
        want.append(oracle.count(s, d, sp.n))
        off = offsets if offsets is not None else (32 if k % 3 else 64)
        graphs.append(tc.preprocess(s, d, sp.n, offsets=off))
    return graphs, want


def test_batch_matches_oracle_and_single_counts(tc):
    specs = small_batch(1, 96)
    graphs, want = build(tc, specs)
    b = tc.Batch(graphs)
    got = b.count().cpu().numpy()
    assert got.tolist() == want
    # the same graphs counted one per launch
    assert [g.count() for g in graphs] == want
    # replaying the captured launch gives the same totals
    assert b.count().cpu().numpy().tolist() == want
    st = b.count_stats()
    assert st["triangles"] == sum(want)
    b.free()
    for g in graphs:
        g.free()


def test_batch_edge_cases(tc):
    specs = [inputs.GraphSpec("gnp", 5, 2, p=0.0),                 # no edges
             inputs.GraphSpec("gnp", 6, 30, p=1.0),                # K_30: warp and CTA units
             inputs.rmat_graph(7, 10, 16)]
    graphs, want = build(tc, specs)
    e = [(a, b) for a in range(200) for b in range(a + 1, 200)]    # K_200
    s = np.array([x for x, _ in e], np.int32)
    d = np.array([y for _, y in e], np.int32)
    graphs.append(tc.preprocess(s, d, 200))
    want.append(200 * 199 * 198 // 6)
    assert tc.count_batch(graphs).cpu().numpy().tolist() == want
    b = tc.Batch(graphs[1:2])   # a batch of one
    assert b.count().cpu().numpy().tolist() == want[1:2]
    b.free()
    for g in graphs:
        g.free()


def test_batch_autotune_keeps_counts(tc):
    specs = small_batch(3, 40, max_log_n=13)
    graphs, want = build(tc, specs, offsets=32)
    b = tc.Batch(graphs)
    t = b.autotune(reps=1)
    assert t.small_max_outdeg in (16, 64) and t.cta_threads in (128, 256)
    assert t.merge_max_outdeg in (0, 16)
    assert b.count().cpu().numpy().tolist() == want
    # a second batch with the same profile reuses the cached choice
    b2 = tc.Batch(graphs)
    t2 = b2.autotune(reps=1)
    assert (t2.small_max_outdeg, t2.warp_unit_tasks, t2.cta_unit_tasks, t2.cta_threads,
            t2.merge_max_outdeg) == \
           (t.small_max_outdeg, t.warp_unit_tasks, t.cta_unit_tasks, t.cta_threads, t.merge_max_outdeg)
    assert b2.count().cpu().numpy().tolist() == want
    for x in (b, b2):
        x.free()
    for g in graphs:
        g.free()


def test_components_union_matches_each_graph(tc):
    """A disjoint union preprocessed once, counted per component."""
    specs = small_batch(5, 30, max_log_n=11)
    srcs, dsts, vpre, want = [], [], [0], []
    for sp in specs:
        s, d = sp.generate()
        want.append(oracle.count(s, d, sp.n))
        srcs.append(s.astype(np.int64) + vpre[-1])
        dsts.append(d.astype(np.int64) + vpre[-1])
        vpre.append(vpre[-1] + sp.n)
    s = np.concatenate(srcs).astype(np.int32)
    d = np.concatenate(dsts).astype(np.int32)
    for dev in (False, True):
        a, b = (torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()) if dev else (s, d)
        g = tc.preprocess_components(a, b, vpre)
        assert tc.count_components(g).cpu().numpy().tolist() == want
        assert g.count() == sum(want)          # the plain count of the union
        g.free()
    # a pair across two components is rejected
    bad_s = np.concatenate([s, np.array([0], np.int32)])
    bad_d = np.concatenate([d, np.array([vpre[-1] - 1], np.int32)])
    with pytest.raises(tc.TCError) as ei:
        tc.preprocess_components(bad_s, bad_d, vpre)
    assert ei.value.status == tc.TC_EINVAL


def test_components_union_on_the_large_input_path(tc):
    """A union of more than 2^26 pairs takes the radix-sort deduplication;
    each component's count still equals that graph counted alone, and a
    pair across two components is still rejected there."""
    parts = [(5, 21, (1 << 25) + 3), (6, 21, 1 << 25)]
    srcs, dsts, vpre, want = [], [], [0], []
    for seed, scale, num in parts:
        s, d = tc.generate_rmat(seed, scale, num)
        g = tc.preprocess(s, d, 1 << scale)
        want.append(g.count())
        g.free()
        srcs.append(s + vpre[-1])
        dsts.append(d + vpre[-1])
        vpre.append(vpre[-1] + (1 << scale))
    s, d = torch.cat(srcs), torch.cat(dsts)
    assert s.shape[0] > (1 << 26)
    g = tc.preprocess_components(s, d, vpre)
    assert tc.count_components(g).cpu().numpy().tolist() == want
    assert g.count() == sum(want)
    g.free()
    s[0] = vpre[1]                       # a pair from component 0 into component 1
    with pytest.raises(tc.TCError) as ei:
        tc.preprocess_components(s, d, vpre)
    assert ei.value.status == tc.TC_EINVAL


GOLDEN_BATCH = os.path.join(os.path.dirname(__file__), "golden", "batch4096_oracle.json")


def test_full_4096_graph_batch_against_stored_oracle(tc):
    """The batched workload at its stated size: all 4096 graphs (half
    G(n,p), half RMAT, n up to 2^16, 8.1e8 pairs) in one autotuned persistent
    launch, every total compared with the oracle's total for that graph,
    stored by tests/golden/make_golden.py --batch.  Then the same graphs as
    one disjoint union (the large-input radix path), counted per component."""
    with open(GOLDEN_BATCH) as f:
        gold = json.load(f)
    num = gold["graphs"]
    graphs, usrc, udst, vpre = [], [], [], [0]
    for g in range(num):
        spec = inputs.batch_member(gold["seed"], g)
        hs, hd = spec.generate()
        assert spec.n == gold["n"][g] and hs.size == gold["num_pairs"][g]
        s, d = torch.from_numpy(hs).cuda(), torch.from_numpy(hd).cuda()
        graphs.append(tc.preprocess(s, d, spec.n, offsets=32))
        usrc.append(s + vpre[-1])
        udst.append(d + vpre[-1])
        vpre.append(vpre[-1] + spec.n)
    assert [g.stats()["m"] for g in graphs] == gold["m"]
    b = tc.Batch(graphs)
    b.autotune(reps=1)
    got = b.count().cpu().numpy().tolist()
    assert got == gold["total"]
    assert b.count_stats()["triangles"] == sum(gold["total"])
    b.free()
    for g in graphs:
        g.free()
    s, d = torch.cat(usrc), torch.cat(udst)
    del usrc, udst
    assert s.shape[0] > (1 << 26)
    gu = tc.preprocess_components(s, d, vpre)
    assert tc.count_components(gu).cpu().numpy().tolist() == gold["total"]
    gu.free()
