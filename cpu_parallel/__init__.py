"""Shared-memory parallel CPU triangle counter (OpenMP) -- a speed baseline.

``tc_openmp.c`` is the paper's shared-memory method (Section 3.1, Eq. 6 and
Eq. 7, enumerated <j,i,k> with the maps of Section 5.2) on all host cores.
It shares no code with the oracle or the CUDA library; ``bench.py`` times it
beside the oracle and the tests check it against the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tc_openmp.c")
_SO = os.path.join(_HERE, "_build", "libtc_openmp.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the counter with gcc -fopenmp into cpu_parallel/_build."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp],
                   check=True)
    os.replace(tmp, _SO)
    return _SO


class _Stats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("max_outdeg", ctypes.c_int64), ("max_deg", ctypes.c_int64),
                ("threads", ctypes.c_int32), ("pad", ctypes.c_int32)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        lib.tcp_count.argtypes = [vp, vp, i64, i64, ctypes.c_int, vp, vp, ctypes.POINTER(_Stats)]
        lib.tcp_count.restype = ctypes.c_int
        _lib = lib
    return _lib


def count(src, dst, n: int, per_vertex: bool = False, threads: int = 0):
    """(total, per-vertex array or None, stats) of the simple undirected graph
    of the pairs; threads = 0 uses every OpenMP thread."""
    s = np.ascontiguousarray(src, dtype=np.int32)
    d = np.ascontiguousarray(dst, dtype=np.int32)
    assert s.shape == d.shape
    total = ctypes.c_uint64(0)
    t = np.zeros(max(n, 1), dtype=np.uint64) if per_vertex else None
    st = _Stats()
    rc = _load().tcp_count(s.ctypes.data, d.ctypes.data, s.shape[0], n, threads,
                           ctypes.addressof(total), t.ctypes.data if per_vertex else None,
                           ctypes.byref(st))
    if rc != 0:
        raise ValueError("cpu_parallel: invalid input (id outside [0, n) or negative size)")
    return (int(total.value), t[:n] if per_vertex else None,
            dict(m=int(st.m), max_outdeg=int(st.max_outdeg), max_deg=int(st.max_deg),
                 threads=int(st.threads)))
