"""CPU oracle for exact triangle counting -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
binding) never imports it, and the two share no code: the oracle is the plain
single-threaded C program ``tc_oracle.c``, which follows the paper's Eq. 1 and
Eq. 2 over a degree-ordered upper-triangular CSR (Sections 3.1 and 5.3), plus
a from-the-definition per-vertex counter for sampled vertices (Section 2).

Every function here is pinned by ``tests/test_oracle.py`` against brute force,
closed forms, invariants and, where installed, networkx.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")


def _so_path(mutant: int = 0) -> str:
    name = "libtc_oracle.so" if mutant == 0 else f"libtc_oracle_mutant{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build; returns the .so path.

    ``mutant`` > 0 compiles a variant with a planted mistake, used only by the
    mutation tests that show the pins catch it."""
    so = _so_path(mutant)
    if (not force and os.path.exists(so)
            and os.path.getmtime(so) >= os.path.getmtime(_SRC)):
        return so
    os.makedirs(_BUILD, exist_ok=True)
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", f"-DTC_ORACLE_MUTANT={mutant}",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


class _Stats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("max_outdeg", ctypes.c_int64),
                ("max_deg", ctypes.c_int64), ("wedges_ijk", ctypes.c_uint64),
                ("wedges_jik", ctypes.c_uint64)]


_libs: dict[int, ctypes.CDLL] = {}


def _lib(mutant: int = 0) -> ctypes.CDLL:
    if mutant in _libs:
        return _libs[mutant]
    lib = ctypes.CDLL(build(mutant))
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.tc_oracle_count.argtypes = [vp, vp, i64, i64, vp, vp, ctypes.POINTER(_Stats)]
    lib.tc_oracle_count.restype = ctypes.c_int
    lib.tc_oracle_vertex_triangles.argtypes = [vp, vp, i64, i64, vp, i64, vp]
    lib.tc_oracle_vertex_triangles.restype = ctypes.c_int
    _libs[mutant] = lib
    return lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def count(src, dst, n: int, per_vertex: bool = False, stats: bool = False,
          mutant: int = 0):
    """Exact triangle count of the simple undirected graph on n vertices whose
    edges are the pairs (src[e], dst[e]) after dropping self-loops and
    duplicates (either direction).

    Returns ``total`` or ``(total, t)`` with t[v] the number of triangles that
    contain original vertex v; with ``stats`` a dict of m, max out-degree,
    max degree and the two enumeration schemes' wedge counts is appended."""
    s, d = _i32(src), _i32(dst)
    assert s.shape == d.shape
    total = ctypes.c_uint64(0)
    t = np.zeros(max(n, 1), dtype=np.uint64) if per_vertex else None
    st = _Stats()
    rc = _lib(mutant).tc_oracle_count(
        s.ctypes.data, d.ctypes.data, s.shape[0], n, ctypes.addressof(total),
        t.ctypes.data if per_vertex else None, ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle: invalid input (id outside [0, n) or negative size)")
    out = [int(total.value)]
    if per_vertex:
        out.append(t[:n])
    if stats:
        out.append(dict(m=int(st.m), max_outdeg=int(st.max_outdeg), max_deg=int(st.max_deg),
                        wedges_ijk=int(st.wedges_ijk), wedges_jik=int(st.wedges_jik)))
    return out[0] if len(out) == 1 else tuple(out)


def vertex_triangles(src, dst, n: int, samples) -> np.ndarray:
    """Triangles through each sampled original vertex (at most 64 samples),
    counted from the definition as edges among its neighbours."""
    s, d = _i32(src), _i32(dst)
    smp = _i32(samples)
    assert smp.shape[0] <= 64
    out = np.zeros(max(smp.shape[0], 1), dtype=np.uint64)
    rc = _lib().tc_oracle_vertex_triangles(s.ctypes.data, d.ctypes.data, s.shape[0], n,
                                           smp.ctypes.data, smp.shape[0], out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle: invalid input")
    return out[:smp.shape[0]]
