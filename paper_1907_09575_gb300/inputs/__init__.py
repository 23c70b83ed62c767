"""Seeded synthetic inputs for the triangle counter.

This module generates the raw pair lists (directed, possibly duplicated,
possibly with self-loops) that ingestion normalises; it holds none of the
counting method's arithmetic.  Both the CPU oracle and the GPU path consume
its output, so both sides see identical bytes.

The workloads mirror the paper's: graph500-style RMAT graphs (Section 6.1,
the g500-s26..s29 rows of the datasets table, a/b/c/d = 0.57/0.19/0.19/0.05)
and, standing in for the skewed twitter / friendster social graphs of the same
table, a Chung-Lu power-law graph.  The real datasets are not used; nothing
here reproduces their contents.

Generator definitions (splitmix64 counter-based draws, RMAT recursion with
integer thresholds, Chung-Lu inverse-CDF sampling, G(n,p) geometric skipping)
are documented in ``gen_host.c``; the GPU library carries an independent device
implementation of the integer RMAT stream, checked bit-for-bit against this one.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen_host.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libtcgen_host.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the host generator (gcc, OpenMP) in-tree; returns the .so path."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u64, i64, i32, u32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32
    vp = ctypes.c_void_p
    lib.tcgen_key.argtypes = [u64, u64]
    lib.tcgen_key.restype = u64
    lib.tcgen_draw.argtypes = [u64, u64]
    lib.tcgen_draw.restype = u64
    lib.tcgen_rmat_scramble_params.argtypes = [u64, i32, vp]
    lib.tcgen_rmat_scramble_params.restype = None
    lib.tcgen_rmat.argtypes = [u64, i32, i64, i64, i64, u32, u32, u32, vp, vp]
    lib.tcgen_rmat.restype = None
    lib.tcgen_chung_lu.argtypes = [u64, vp, i64, i64, i64, vp, vp]
    lib.tcgen_chung_lu.restype = None
    lib.tcgen_gnp.argtypes = [u64, i64, ctypes.c_double, vp, vp, i64]
    lib.tcgen_gnp.restype = i64
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# ----------------------------------------------------------------------------
# primitive streams
# ----------------------------------------------------------------------------

def key(seed: int, tag: int) -> int:
    return int(_load().tcgen_key(seed & (2**64 - 1), tag))


def draw(k: int, ctr: int) -> int:
    return int(_load().tcgen_draw(k, ctr))


def uniform01(seed: int, tag: int, ctr: int) -> float:
    """A double in [0, 1) from the top 53 bits of one draw."""
    return (draw(key(seed, tag), ctr) >> 11) * 2.0 ** -53


def rmat_thresholds(a: str = "0.57", b: str = "0.19", c: str = "0.19") -> tuple[int, int, int]:
    """Cumulative a, a+b, a+b+c as exact floor(x * 2^32) integers."""
    fa, fb, fc = Fraction(a), Fraction(b), Fraction(c)
    s = 2 ** 32
    return (math.floor(fa * s), math.floor((fa + fb) * s), math.floor((fa + fb + fc) * s))


def rmat_scramble_params(seed: int, scale: int) -> tuple[int, int, int]:
    out = np.zeros(3, dtype=np.uint64)
    _load().tcgen_rmat_scramble_params(seed, scale, _ptr(out))
    return int(out[0]), int(out[1]), int(out[2])


def rmat(seed: int, scale: int, num_pairs: int, n: int | None = None,
         thresholds: tuple[int, int, int] | None = None,
         e0: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Pairs [e0, e0 + num_pairs) of the RMAT stream of (seed, scale, n)."""
    if n is None:
        n = 1 << scale
    assert 0 < n <= (1 << scale) and scale <= 31
    t1, t2, t3 = thresholds or rmat_thresholds()
    src = np.empty(num_pairs, dtype=np.int32)
    dst = np.empty(num_pairs, dtype=np.int32)
    if num_pairs:
        _load().tcgen_rmat(seed, scale, n, e0, num_pairs, t1, t2, t3, _ptr(src), _ptr(dst))
    return src, dst


def chung_lu_weights(n: int, gamma: float = 2.1, mean_degree: float = 40.0,
                     wmax: float = 1e6, i0: int = 1,
                     weight_scale: float = 65536.0) -> np.ndarray:
    """Inclusive prefix sums of integer Chung-Lu weights.

    Expected degree w_i = min(c * (i + i0)^(-1/(gamma-1)), wmax), with c found
    by bisection so that the mean of w is ``mean_degree`` after capping; the
    integer weight is round(w_i * weight_scale)."""
    x = np.arange(n, dtype=np.float64) + float(i0)
    base = x ** (-1.0 / (gamma - 1.0))

    def mean_w(c: float) -> float:
        return float(np.minimum(c * base, wmax).mean())

    lo, hi = 0.0, 1.0
    while mean_w(hi) < mean_degree:
        hi *= 2.0
        if hi > 1e300:
            raise ValueError("mean degree unreachable under the cap")
    for _ in range(64):   # halves the bracket each time: far below one ulp of c
        mid = 0.5 * (lo + hi)
        if mean_w(mid) < mean_degree:
            lo = mid
        else:
            hi = mid
    w = np.minimum(hi * base, wmax)
    iw = np.rint(w * weight_scale).astype(np.uint64)
    iw[iw == 0] = 1
    return np.cumsum(iw, dtype=np.uint64)


def chung_lu(seed: int, cum: np.ndarray, num_pairs: int, e0: int = 0) -> tuple[np.ndarray, np.ndarray]:
    cum = np.ascontiguousarray(cum, dtype=np.uint64)
    n = cum.shape[0]
    src = np.empty(num_pairs, dtype=np.int32)
    dst = np.empty(num_pairs, dtype=np.int32)
    if num_pairs:
        _load().tcgen_chung_lu(seed, _ptr(cum), n, e0, num_pairs, _ptr(src), _ptr(dst))
    return src, dst


def gnp(seed: int, n: int, p: float) -> tuple[np.ndarray, np.ndarray]:
    cap = max(16, int(p * n * (n - 1) / 2 * 1.2) + 64)
    while True:
        src = np.empty(cap, dtype=np.int32)
        dst = np.empty(cap, dtype=np.int32)
        cnt = int(_load().tcgen_gnp(seed, n, p, _ptr(src), _ptr(dst), cap))
        if cnt <= cap:
            return src[:cnt].copy(), dst[:cnt].copy()
        cap = cnt


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class GraphSpec:
    """A reproducible synthetic graph: kind, seed, vertex count and pair count."""
    kind: str            # "rmat" | "chung_lu" | "gnp"
    seed: int
    n: int
    num_pairs: int = 0   # rmat / chung_lu
    scale: int = 0       # rmat
    p: float = 0.0       # gnp
    gamma: float = 2.1   # chung_lu
    mean_degree: float = 40.0
    wmax: float = 1e6

    def generate(self) -> tuple[np.ndarray, np.ndarray]:
        if self.kind == "rmat":
            return rmat(self.seed, self.scale, self.num_pairs, n=self.n)
        if self.kind == "chung_lu":
            cum = chung_lu_weights(self.n, self.gamma, self.mean_degree, self.wmax)
            return chung_lu(self.seed, cum, self.num_pairs)
        if self.kind == "gnp":
            return gnp(self.seed, self.n, self.p)
        raise ValueError(self.kind)


def rmat_graph(seed: int, scale: int, edge_factor: int = 16) -> GraphSpec:
    """graph500-shaped RMAT: n = 2^scale, edge_factor * n generated pairs."""
    n = 1 << scale
    return GraphSpec("rmat", seed, n, num_pairs=edge_factor * n, scale=scale)


def chung_lu_graph(seed: int, n: int = 50_000_000, gamma: float = 2.1,
                   mean_degree: float = 40.0, wmax: float = 1e6) -> GraphSpec:
    """Chung-Lu power law: n * mean_degree / 2 pairs drawn by weight."""
    return GraphSpec("chung_lu", seed, n, num_pairs=int(n * mean_degree / 2),
                     gamma=gamma, mean_degree=mean_degree, wmax=wmax)


TAG_BATCH = 0x42415443   # "BATC"
TAG_SERVE = 0x53525645   # "SRVE"


def batch_member(seed: int, g: int) -> GraphSpec:
    """Graph g of the uneven batch: even g -> G(n,p), odd g -> RMAT.

    n = floor(2^(8 + 8 U1)), mean degree d = 4 + 60 U2 with U1, U2 uniforms
    drawn from the batch stream; G(n,p) uses p = d/(n-1); RMAT draws n*d/2
    pairs at scale ceil(log2 n), rejecting ids >= n."""
    k = key(seed, TAG_BATCH)
    u1 = (draw(k, 4 * g) >> 11) * 2.0 ** -53
    u2 = (draw(k, 4 * g + 1) >> 11) * 2.0 ** -53
    gseed = draw(k, 4 * g + 2)
    n = int(math.floor(2.0 ** (8.0 + 8.0 * u1)))
    n = max(2, min(n, 1 << 16))
    d = 4.0 + 60.0 * u2
    if g % 2 == 0:
        return GraphSpec("gnp", gseed, n, p=min(1.0, d / (n - 1)))
    scale = max(1, math.ceil(math.log2(n)))
    return GraphSpec("rmat", gseed, n, num_pairs=int(n * d / 2), scale=scale)


def serve_request(seed: int, r: int) -> GraphSpec:
    """Request r of the served stream: M = floor(2^(10 + 12 U)) pairs,
    edge factor e uniform in [8, 32], n = ceil(M / e), RMAT at scale
    ceil(log2 n) with ids >= n rejected."""
    k = key(seed, TAG_SERVE)
    u = (draw(k, 4 * r) >> 11) * 2.0 ** -53
    e = 8 + int(draw(k, 4 * r + 1) % 25)
    rseed = draw(k, 4 * r + 2)
    m = int(math.floor(2.0 ** (10.0 + 12.0 * u)))
    n = max(2, -(-m // e))
    scale = max(1, math.ceil(math.log2(n)))
    return GraphSpec("rmat", rseed, n, num_pairs=m, scale=scale)


def serve_arrivals(seed: int, rate_hz: float, duration_s: float) -> np.ndarray:
    """Poisson arrival times (seconds) of an open-loop stream at rate_hz."""
    k = key(seed, TAG_SERVE + 1)
    t, out, i = 0.0, [], 0
    while True:
        u = ((draw(k, i) >> 11) + 1) * 2.0 ** -53
        i += 1
        t += -math.log(u) / rate_hz
        if t >= duration_s:
            return np.asarray(out, dtype=np.float64)
        out.append(t)
