"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Counts are integers, so the bar is bit-exact equality of the total and of
every per-vertex count.  Inputs are seeded synthetic graphs from
``paper_1907_09575_gb300.inputs`` (host generated, uploaded) plus hand-built
edge cases; expected values come only from ``oracle`` or closed forms.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1907_09575_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tc():
    from paper_1907_09575_gb300 import tc as _tc
    _tc.load()
    return _tc


def gpu_count(tc, src, dst, n, per_vertex=True, device_input=True, offsets=None, tuning=None):
    s = np.ascontiguousarray(src, dtype=np.int32)
    d = np.ascontiguousarray(dst, dtype=np.int32)
    if device_input:
        g = tc.preprocess(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n, offsets=offsets)
    else:
        g = tc.preprocess(s, d, n, offsets=offsets)
    try:
        if per_vertex:
            total, t = g.count(per_vertex=True, tuning=tuning)
            return total, t.cpu().numpy().astype(np.uint64), g.stats()
        return g.count(tuning=tuning), None, g.stats()
    finally:
        g.free()


def check(tc, src, dst, n, **kw):
    want, want_t, st = oracle.count(src, dst, n, per_vertex=True, stats=True)
    got, got_t, gst = gpu_count(tc, src, dst, n, **kw)
    assert got == want
    if got_t is not None:
        assert np.array_equal(got_t[:n], want_t)
    assert gst["m"] == st["m"]
    assert gst["max_outdeg"] == st["max_outdeg"]
    assert gst["max_deg"] == st["max_deg"]
    assert gst["probes"] == st["wedges_jik"]
    assert gst["probes_ijk"] == st["wedges_ijk"]
    return want


def edges_to_arrays(e):
    if not e:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    a = np.asarray(e, dtype=np.int64)
    return a[:, 0].astype(np.int32), a[:, 1].astype(np.int32)


# ----------------------------------------------------------------------------
# device generator = host generator, bit for bit
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed,scale,n,num", [(1, 14, None, 262144), (7, 10, 700, 50000),
                                              (3, 20, None, 100000), (9, 1, 2, 1000),
                                              (2, 26, None, 65536)])
def test_device_generator_matches_host(tc, seed, scale, n, num):
    hs, hd = inputs.rmat(seed, scale, num, n=n)
    ds, dd = tc.generate_rmat(seed, scale, num, n=n)
    assert np.array_equal(ds.cpu().numpy(), hs)
    assert np.array_equal(dd.cpu().numpy(), hd)
    # a slice from the middle of the stream
    hs2, hd2 = inputs.rmat(seed, scale, 1000, n=n, e0=12345)
    ds2, dd2 = tc.generate_rmat(seed, scale, 1000, n=n, e0=12345)
    assert np.array_equal(ds2.cpu().numpy(), hs2) and np.array_equal(dd2.cpu().numpy(), hd2)


# ----------------------------------------------------------------------------
# edge cases and closed forms
# ----------------------------------------------------------------------------

def test_empty_inputs(tc):
    for n in (0, 1, 5):
        total, t, st = gpu_count(tc, [], [], n)
        assert total == 0 and st["m"] == 0
        assert t is None or np.all(t[:n] == 0)
    # only self-loops
    total, t, st = gpu_count(tc, [0, 1, 2, 2], [0, 1, 2, 2], 3)
    assert total == 0 and st["m"] == 0


def test_single_edge_and_triangle(tc):
    assert gpu_count(tc, [0], [1], 2)[0] == 0
    total, t, _ = gpu_count(tc, [0, 1, 2], [1, 2, 0], 3)
    assert total == 1 and t.tolist() == [1, 1, 1]
    # same triangle given twice in both directions with loops
    total, t, _ = gpu_count(tc, [0, 1, 2, 1, 2, 0, 1], [1, 2, 0, 0, 1, 2, 1], 3)
    assert total == 1 and t.tolist() == [1, 1, 1]


@pytest.mark.parametrize("n", [3, 4, 5, 33, 64, 65, 66, 130, 300])
def test_complete_graphs(tc, n):
    e = [(a, b) for a in range(n) for b in range(a + 1, n)]
    s, d = edges_to_arrays(e)
    total, t, _ = gpu_count(tc, s, d, n)
    assert total == math.comb(n, 3)
    assert np.all(t[:n] == math.comb(n - 1, 2))


@pytest.mark.parametrize("n", [4, 5, 8, 70, 1000])
def test_wheels(tc, n):
    rim = list(range(1, n))
    e = [(0, r) for r in rim] + [(rim[i], rim[(i + 1) % len(rim)]) for i in range(len(rim))]
    s, d = edges_to_arrays(e)
    total, t, _ = gpu_count(tc, s, d, n)
    if n == 4:
        assert total == 4
    else:
        assert total == n - 1 and t[0] == n - 1 and np.all(t[1:n] == 2)


def test_counting_csr_row_lengths(tc):
    # a planted K_601 on random vertices among RMAT edges, in shuffled order:
    # rows of U of every length up to 600 reach every sort of the counting
    # CSR build (one, two, four or eight entries a lane; a block above 256)
    rng = np.random.default_rng(11)
    n = 4096
    hs, hd = inputs.rmat(5, 12, 30000)
    core = rng.choice(n, 601, replace=False).astype(np.int32)
    iu, ju = np.triu_indices(601, 1)
    src = np.concatenate([hs, core[iu]])
    dst = np.concatenate([hd, core[ju]])
    order = rng.permutation(src.size)
    check(tc, src[order], dst[order], n)
    _, _, st = gpu_count(tc, src[order], dst[order], n, per_vertex=False)
    assert st["max_outdeg"] >= 600


def test_bipartite_star_cycle(tc):
    rng = np.random.default_rng(0)
    e = [(x, 60 + y) for x in range(60) for y in range(50) if rng.random() < 0.4]
    s, d = edges_to_arrays(e)
    assert gpu_count(tc, s, d, 110)[0] == 0
    s, d = edges_to_arrays([(0, v) for v in range(1, 5000)])
    assert gpu_count(tc, s, d, 5000)[0] == 0
    s, d = edges_to_arrays([(v, (v + 1) % 999) for v in range(999)])
    assert gpu_count(tc, s, d, 999)[0] == 0


def test_textbook_graphs(tc):
    with open(os.path.join(GOLDEN, "textbook_graphs.json")) as f:
        graphs = json.load(f)
    for g in graphs:
        s, d = edges_to_arrays(g["edges"])
        total, t, _ = gpu_count(tc, s, d, g["n"])
        assert total == g["total"], g["name"]
        assert t[: g["n"]].tolist() == g["per_vertex"], g["name"]


def test_invalid_ids_rejected(tc):
    with pytest.raises(tc.TCError) as ei:
        gpu_count(tc, [0, 1, 7], [1, 2, 0], 5)
    assert ei.value.status == tc.TC_EINVAL
    with pytest.raises(tc.TCError):
        gpu_count(tc, [-1], [0], 5)
    # the library stays usable afterwards
    assert gpu_count(tc, [0, 1, 2], [1, 2, 0], 3)[0] == 1


# ----------------------------------------------------------------------------
# random graphs, both offset widths, host and device input
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(10))
def test_random_graphs(tc, seed):
    rng = np.random.default_rng(seed)
    kind = seed % 3
    if kind == 0:
        spec = inputs.rmat_graph(seed + 1, int(rng.integers(6, 13)), int(rng.integers(2, 24)))
    elif kind == 1:
        spec = inputs.GraphSpec("gnp", seed + 1, int(rng.integers(10, 3000)),
                                p=float(rng.uniform(0.001, 0.2)))
    else:
        cum = inputs.chung_lu_weights(5000, 2.1, 12.0, 400.0)
        s, d = inputs.chung_lu(seed, cum, 30000)
        check(tc, s, d, 5000, offsets=[None, 32, 64][seed % 3], device_input=bool(seed % 2))
        return
    s, d = spec.generate()
    check(tc, s, d, spec.n, offsets=[None, 32, 64][seed % 3], device_input=bool(seed % 2))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rmat_scale14_golden(tc, seed):
    """The small single-graph workload: RMAT scale 14, edge factor 16, int32
    offsets, total count; compared with the stored oracle result and live."""
    with open(os.path.join(GOLDEN, "rmat_s14_oracle.json")) as f:
        gold = json.load(f)[str(seed)]
    spec = inputs.rmat_graph(seed, 14, 16)
    s, d = tc.generate_rmat(seed, 14, spec.num_pairs)
    g = tc.preprocess(s, d, spec.n, offsets=32)
    assert g.count() == gold["total"]
    st = g.stats()
    assert st["m"] == gold["m"] and st["offset_bytes"] == 4
    assert st["probes"] == gold["wedges_jik"]
    g.free()
    hs, hd = spec.generate()
    check(tc, hs, hd, spec.n, offsets=32)


# ----------------------------------------------------------------------------
# every kernel path forced, same answers
# ----------------------------------------------------------------------------

TUNINGS = [
    dict(),
    dict(small_max_outdeg=1),                      # everything through the CTA kernel
    dict(small_max_outdeg=64, slice_max=64),       # pivots split into many slices
    dict(warp_unit_tasks=1, cta_unit_tasks=1),     # one task per unit
    dict(cta_threads=256, cta_unit_tasks=100000),  # one unit per pivot (tasks capped at 8192)
    dict(cta_threads=64, slice_max=100),
    dict(table_mode=1),                            # hash tables only
    dict(table_mode=1, small_max_outdeg=1, slice_max=64),
    dict(merge_max_outdeg=64),                     # every warp unit by search, no table
    dict(merge_max_outdeg=8, small_max_outdeg=16, warp_unit_tasks=3),
]


@pytest.mark.parametrize("ti", range(len(TUNINGS)))
def test_kernel_paths_agree(tc, ti):
    t = tc.Tuning()
    for k, v in TUNINGS[ti].items():
        setattr(t, k, v)
    # a hub-heavy graph: RMAT plus a vertex adjacent to a third of the rest
    spec = inputs.rmat_graph(5, 13, 16)
    s, d = spec.generate()
    hub = np.full(spec.n // 3, 17, dtype=np.int32)
    others = np.arange(0, spec.n, 3, dtype=np.int32)[: hub.size]
    s = np.concatenate([s, hub])
    d = np.concatenate([d, others])
    check(tc, s, d, spec.n, tuning=t)
    # complete graph with pivots above the warp limit
    e = [(a, b) for a in range(150) for b in range(a + 1, 150)]
    s2, d2 = edges_to_arrays(e)
    total, tv, _ = gpu_count(tc, s2, d2, 150, tuning=t)
    assert total == math.comb(150, 3) and np.all(tv[:150] == math.comb(149, 2))


def test_repeatable(tc):
    spec = inputs.rmat_graph(2, 15, 16)
    s, d = tc.generate_rmat(2, 15, spec.num_pairs)
    g = tc.preprocess(s, d, spec.n)
    res = [g.count() for _ in range(5)]
    pv = [g.count(per_vertex=True)[1].cpu().numpy() for _ in range(3)]
    assert len(set(res)) == 1
    assert all(np.array_equal(pv[0], x) for x in pv[1:])
    g.free()


def test_one_shot_host_call(tc):
    spec = inputs.rmat_graph(4, 12, 16)
    s, d = spec.generate()
    want, want_t = oracle.count(s, d, spec.n, per_vertex=True)
    total, t = tc.triangles(s, d, spec.n, per_vertex=True)
    assert total == want and np.array_equal(t, want_t)
    assert tc.triangles(s, d, spec.n) == want


@pytest.mark.parametrize("num", [1, 2, 4095, 4096, 4097, 8191, 8192, 12289, 65535, 65537, 262143])
def test_sort_tile_boundaries(tc, num):
    """Pair counts around multiples of the 4096-key sort tile (one tile, a
    ragged last tile, many tiles) for random and RMAT-shaped graphs."""
    rng = np.random.default_rng(num)
    n = int(max(2, min(num, 5000)))
    s = rng.integers(0, n, size=num).astype(np.int32)
    d = rng.integers(0, n, size=num).astype(np.int32)
    check(tc, s, d, n)
    hs, hd = inputs.rmat(num, 12, num)
    check(tc, hs, hd, 4096, offsets=64)


def test_dedup_paths_agree(tc):
    """Inputs up to 2^26 pairs are deduplicated through a hash set, larger
    ones by the radix sort.  The same pairs given twice cross that bound
    without changing the graph: both paths must build the same graph and
    counts, and sampled vertices must match the oracle."""
    num = (1 << 25) + 1000
    s, d = tc.generate_rmat(11, 21, num)
    s2, d2 = torch.cat([s, d]), torch.cat([d, s])          # every pair again, reversed
    assert s.shape[0] <= (1 << 26) < s2.shape[0]
    n = 1 << 21
    out = []
    for a, b in ((s, d), (s2, d2)):
        g = tc.preprocess(a, b, n)
        total, t = g.count(per_vertex=True)
        out.append((total, t.cpu().numpy(), g.stats()))
        g.free()
    (t1, pv1, st1), (t2, pv2, st2) = out
    assert t1 == t2 and np.array_equal(pv1, pv2)
    for k in ("m", "max_deg", "max_outdeg", "tasks", "probes", "probes_ijk"):
        assert st1[k] == st2[k], k
    assert int(pv1.sum()) == 3 * t1
    hs, hd = inputs.rmat(11, 21, num)
    deg = np.bincount(hs, minlength=n) + np.bincount(hd, minlength=n)
    rng = np.random.default_rng(5)
    pick = rng.choice(np.flatnonzero((deg > 2) & (deg < 300)), size=24, replace=False).astype(np.int32)
    want = oracle.vertex_triangles(hs, hd, n, pick)
    assert np.array_equal(pv1[pick].astype(np.uint64), want)


def test_invalid_id_on_the_sort_path(tc):
    """Inputs above 2^26 pairs take the radix-sort deduplication; an id
    outside [0, n) there is reported too, and the library stays usable."""
    num = (1 << 26) + 10
    n = 1 << 20
    s, d = tc.generate_rmat(3, 20, num)
    s[num // 2] = n + 5
    with pytest.raises(tc.TCError) as ei:
        tc.preprocess(s, d, n)
    assert ei.value.status == tc.TC_EINVAL
    s[num // 2] = 0
    g = tc.preprocess(s, d, n)
    assert g.stats()["m"] > 0 and g.count() > 0
    g.free()


def test_pinned_host_input_paths(tc):
    """Host pairs in page-locked memory are uploaded by SM loads (vector or,
    for a buffer not 16-byte aligned, scalar); pageable ones by the copy
    engine.  All give the oracle's counts, through tc_preprocess and
    tc_triangles."""
    spec = inputs.rmat_graph(4, 15, 16)
    hs, hd = spec.generate()
    want, want_t = oracle.count(hs, hd, spec.n, per_vertex=True)
    ps = torch.empty(hs.size + 1, dtype=torch.int32, pin_memory=True)
    pd = torch.empty(hd.size + 1, dtype=torch.int32, pin_memory=True)
    for off in (0, 1):                     # aligned, then one element in
        ps[off:off + hs.size] = torch.from_numpy(hs)
        pd[off:off + hd.size] = torch.from_numpy(hd)
        a = ps[off:off + hs.size].numpy()
        b = pd[off:off + hd.size].numpy()
        g = tc.preprocess(a, b, spec.n)
        total, t = g.count(per_vertex=True)
        g.free()
        assert total == want and np.array_equal(t.cpu().numpy().astype(np.uint64), want_t)
        total2, t2 = tc.triangles(a, b, spec.n, per_vertex=True)
        assert total2 == want and np.array_equal(t2.astype(np.uint64), want_t)
        tm = tc.triangles_timing()
        assert tm["input_pinned"] and tm["h2d_ms"] >= 0 and tm["count_ms"] > 0
    total3 = tc.triangles(hs, hd, spec.n)   # pageable
    assert total3 == want and not tc.triangles_timing()["input_pinned"]
