"""Python binding of the C ABI in ``include/tc.h`` (argument marshalling only).

Every step of preprocessing and counting runs in the CUDA library
``_build/libtc.so``; this module only converts tensors to pointers, passes
the current torch CUDA stream, and turns status codes into exceptions.  There
is no CPU fallback: if the library is missing, loading fails loudly.

Names follow the C functions: ``preprocess`` -> ``tc_preprocess``,
``Graph.count`` -> ``tc_count``, ``triangles`` -> ``tc_triangles``,
``generate_rmat`` -> ``tc_generate_rmat``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libtc.so")

TC_OK, TC_EINVAL, TC_ENOMEM, TC_ECUDA, TC_ETIMEOUT, TC_EBUSY, TC_EUNSUPPORTED = range(7)
TC_INPUT_ON_DEVICE = 0x1
TC_OFFSETS_32 = 0x2
TC_OFFSETS_64 = 0x4

_STATUS = {1: "TC_EINVAL", 2: "TC_ENOMEM", 3: "TC_ECUDA", 4: "TC_ETIMEOUT", 5: "TC_EBUSY",
           6: "TC_EUNSUPPORTED"}


class TCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Tuning(ctypes.Structure):
    _fields_ = [("small_max_outdeg", ctypes.c_int32), ("warp_unit_tasks", ctypes.c_int32),
                ("cta_unit_tasks", ctypes.c_int32), ("cta_threads", ctypes.c_int32),
                ("slice_max", ctypes.c_int32), ("table_mode", ctypes.c_int32),
                ("merge_max_outdeg", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GraphStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("num_pairs", ctypes.c_int64), ("m", ctypes.c_int64),
                ("max_deg", ctypes.c_int64), ("max_outdeg", ctypes.c_int64),
                ("tasks", ctypes.c_int64), ("probes", ctypes.c_uint64),
                ("small_units", ctypes.c_int64), ("large_units", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("offset_bytes", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("probes_ijk", ctypes.c_uint64)]


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                           ctypes.c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                          ctypes.c_void_p)),
                ("ctx", ctypes.c_void_p)]


_lib: Optional[ctypes.CDLL] = None

# Every symbol include/tc.h declares (checked by the tests).
EXPORTS = ("tc_preprocess", "tc_count", "tc_triangles", "tc_graph_get_stats", "tc_graph_free",
           "tc_tuning_default", "tc_last_error", "tc_generate_rmat", "tc_kernel_launches",
           "tc_profile_enable", "tc_profile_read", "tc_count_get_stats", "tc_triangles_static",
           "tc_batch_create", "tc_batch_count", "tc_batch_autotune", "tc_batch_get_count_stats",
           "tc_batch_free", "tc_count_batch", "tc_preprocess_components", "tc_count_components",
           "tc_server_create", "tc_server_now", "tc_server_submit_rmat", "tc_server_poll",
           "tc_server_drain", "tc_server_get_stats", "tc_server_free", "tc_release_memory",
           "tc_selftest_wait_timeout", "tc_server_submit_rmat_many", "tc_memory_get_stats",
           "tc_triangles_get_timing", "tc_graph_offload", "tc_count_tiled")

TC_STATIC_MAX_PAIRS = 262144
TC_STATIC_MAX_VERTICES = 65536


class CountStats(ctypes.Structure):
    _fields_ = [("triangles", ctypes.c_uint64), ("units", ctypes.c_uint64 * 2),
                ("tasks", ctypes.c_uint64 * 2), ("probes", ctypes.c_uint64 * 2),
                ("staged", ctypes.c_uint64 * 2)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("workers", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_tick_pairs", ctypes.c_int64),
                ("device", ctypes.c_int32), ("pad", ctypes.c_int32)]


class RmatSpec(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("scale", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("n", ctypes.c_int64), ("num_pairs", ctypes.c_int64), ("t1", ctypes.c_uint32),
                ("t2", ctypes.c_uint32), ("t3", ctypes.c_uint32), ("pad2", ctypes.c_uint32)]


class ServerResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("triangles", ctypes.c_uint64),
                ("t_arrival", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("status", ctypes.c_int32),
                ("tick_requests", ctypes.c_int32), ("tick_pairs", ctypes.c_int64),
                ("t_dev_start", ctypes.c_double), ("t_dev_end", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "failed", "pending", "ticks",
                                               "bytes_in_flight", "peak_bytes_in_flight",
                                               "busy_workers")] + \
               [("device_busy_s", ctypes.c_double), ("device_overlap_s", ctypes.c_double)]


class MemoryStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("reserved", "reserved_high", "used", "used_high")]


class TrianglesTiming(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in ("wall_ms", "h2d_ms", "preprocess_ms", "count_ms",
                                                "d2h_ms", "h2d_issue_ms")] + \
               [("input_pinned", ctypes.c_int32), ("upload_method", ctypes.c_int32),
                ("ce_slice_gbs", ctypes.c_double), ("sm_slice_gbs", ctypes.c_double)]


class TiledStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("pivot_blocks", "row_blocks", "tiles", "tile_tasks",
                                               "h2d_bytes")] + [("probes", ctypes.c_uint64),
                                                                ("split_pivots", ctypes.c_int64)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (no fallback: raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as "
                           "g; g.build()'` (the CUDA library is required; there is no CPU path)")
    lib = ctypes.CDLL(path)
    vp, i64, u32, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64
    st = ctypes.c_int
    lib.tc_preprocess.argtypes = [vp, vp, i64, i64, u32, vp, vp, ctypes.POINTER(vp)]
    lib.tc_preprocess.restype = st
    lib.tc_count.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.tc_count.restype = st
    lib.tc_triangles.argtypes = [vp, vp, i64, i64, u32, vp, vp, vp]
    lib.tc_triangles.restype = st
    lib.tc_graph_get_stats.argtypes = [vp, ctypes.POINTER(GraphStats)]
    lib.tc_graph_get_stats.restype = st
    lib.tc_graph_free.argtypes = [vp]
    lib.tc_graph_free.restype = None
    lib.tc_selftest_wait_timeout.argtypes = [ctypes.c_int64, vp]
    lib.tc_selftest_wait_timeout.restype = st
    lib.tc_release_memory.argtypes = [ctypes.c_int]
    lib.tc_release_memory.restype = st
    lib.tc_tuning_default.argtypes = [ctypes.POINTER(Tuning)]
    lib.tc_tuning_default.restype = st
    lib.tc_last_error.argtypes = []
    lib.tc_last_error.restype = ctypes.c_char_p
    lib.tc_generate_rmat.argtypes = [u64, i32, i64, i64, i64, u32, u32, u32, vp, vp, vp]
    lib.tc_generate_rmat.restype = st
    lib.tc_count_get_stats.argtypes = [vp, ctypes.POINTER(CountStats), vp]
    lib.tc_count_get_stats.restype = st
    lib.tc_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.tc_server_create.restype = st
    lib.tc_server_now.argtypes = [vp]
    lib.tc_server_now.restype = ctypes.c_double
    lib.tc_server_submit_rmat.argtypes = [vp, ctypes.POINTER(RmatSpec), ctypes.c_double,
                                          ctypes.POINTER(i64)]
    lib.tc_server_submit_rmat.restype = st
    lib.tc_server_submit_rmat_many.argtypes = [vp, ctypes.POINTER(RmatSpec), i32,
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.tc_server_submit_rmat_many.restype = st
    lib.tc_memory_get_stats.argtypes = [ctypes.c_int, i32, ctypes.POINTER(MemoryStats)]
    lib.tc_memory_get_stats.restype = st
    lib.tc_triangles_get_timing.argtypes = [ctypes.POINTER(TrianglesTiming)]
    lib.tc_triangles_get_timing.restype = st
    lib.tc_graph_offload.argtypes = [vp, vp]
    lib.tc_graph_offload.restype = st
    lib.tc_count_tiled.argtypes = [vp, i64, vp, vp, vp, vp, ctypes.POINTER(TiledStats), vp]
    lib.tc_count_tiled.restype = st
    lib.tc_server_poll.argtypes = [vp, ctypes.POINTER(ServerResult), i32, ctypes.POINTER(i32), i32]
    lib.tc_server_poll.restype = st
    lib.tc_server_drain.argtypes = [vp, i32]
    lib.tc_server_drain.restype = st
    lib.tc_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.tc_server_get_stats.restype = st
    lib.tc_server_free.argtypes = [vp]
    lib.tc_server_free.restype = None
    lib.tc_preprocess_components.argtypes = [vp, vp, i64, vp, i32, u32, vp, vp, ctypes.POINTER(vp)]
    lib.tc_preprocess_components.restype = st
    lib.tc_count_components.argtypes = [vp, vp, vp, vp]
    lib.tc_count_components.restype = st
    lib.tc_batch_create.argtypes = [vp, i32, vp, vp, ctypes.POINTER(vp)]
    lib.tc_batch_create.restype = st
    lib.tc_batch_count.argtypes = [vp, vp, vp]
    lib.tc_batch_count.restype = st
    lib.tc_batch_autotune.argtypes = [vp, i32, ctypes.POINTER(Tuning), vp]
    lib.tc_batch_autotune.restype = st
    lib.tc_batch_get_count_stats.argtypes = [vp, ctypes.POINTER(CountStats), vp]
    lib.tc_batch_get_count_stats.restype = st
    lib.tc_batch_free.argtypes = [vp]
    lib.tc_batch_free.restype = None
    lib.tc_count_batch.argtypes = [vp, i32, vp, vp, vp]
    lib.tc_count_batch.restype = st
    lib.tc_triangles_static.argtypes = [vp, vp, i64, i64, vp, vp, vp]
    lib.tc_triangles_static.restype = st
    lib.tc_kernel_launches.argtypes = []
    lib.tc_kernel_launches.restype = ctypes.c_longlong
    lib.tc_profile_enable.argtypes = [i32]
    lib.tc_profile_enable.restype = None
    lib.tc_profile_read.argtypes = [ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)]
    lib.tc_profile_read.restype = st
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != TC_OK:
        msg = load().tc_last_error()
        raise TCError(status, msg.decode() if msg else "")


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x) -> tuple[int, bool]:
    """(address, on_device) of a contiguous int32 torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        assert x.dtype == np.int32 and x.flags["C_CONTIGUOUS"], "need contiguous int32"
        return x.ctypes.data, False
    import torch
    if isinstance(x, torch.Tensor):
        assert x.dtype == torch.int32 and x.is_contiguous(), "need contiguous int32"
        return x.data_ptr(), x.is_cuda
    raise TypeError(type(x))


def kernel_launches() -> int:
    """Kernels this library has launched since it was loaded."""
    return int(load().tc_kernel_launches())


def profile_enable(on: bool = True) -> None:
    """Start (clearing old records) or stop CUDA-event timing of every launch."""
    load().tc_profile_enable(1 if on else 0)


def profile_read() -> dict:
    """{kernel name: (launches, total device ms)} since profiling was enabled."""
    cnt = ctypes.c_int32(0)
    _check(load().tc_profile_read(None, 0, ctypes.byref(cnt)))
    buf = (KernelTime * max(cnt.value, 1))()
    _check(load().tc_profile_read(buf, cnt.value, ctypes.byref(cnt)))
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
            for i in range(cnt.value)}


def selftest_wait_timeout(spin_limit: int = 4096, stream=None) -> int:
    """tc_selftest_wait_timeout: the status of a bounded device wait made to
    run out (TC_ETIMEOUT when the bound works)."""
    return int(load().tc_selftest_wait_timeout(spin_limit, _stream_ptr(stream)))


def release_memory(device: int = -1) -> None:
    """tc_release_memory: give back the device memory the library's pool keeps
    for reuse (device -1: every device)."""
    _check(load().tc_release_memory(device))


def memory_stats(device: int = 0, reset_high: bool = False) -> dict:
    """tc_memory_get_stats: bytes reserved and in use in the library's pool of
    `device`, with their high-water marks (zeroed after reading if reset_high)."""
    m = MemoryStats()
    _check(load().tc_memory_get_stats(device, 1 if reset_high else 0, ctypes.byref(m)))
    return {f: int(getattr(m, f)) for f, _ in MemoryStats._fields_}


def tuning_default() -> Tuning:
    t = Tuning()
    _check(load().tc_tuning_default(ctypes.byref(t)))
    return t


class Graph:
    """A preprocessed graph (owns the library's device arena)."""

    def __init__(self, handle: int, n: int):
        self._h = ctypes.c_void_p(handle)
        self.n = n

    @property
    def handle(self) -> int:
        return self._h.value or 0

    def free(self) -> None:
        if self._h.value:
            load().tc_graph_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self) -> dict:
        s = GraphStats()
        _check(load().tc_graph_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in GraphStats._fields_ if f != "pad"}

    def count_stats(self, stream=None) -> dict:
        """Work counters of the last count (tc_count_get_stats)."""
        c = CountStats()
        _check(load().tc_count_get_stats(self._h, ctypes.byref(c), _stream_ptr(stream)))
        return {"triangles": int(c.triangles), "units": list(c.units), "tasks": list(c.tasks),
                "probes": list(c.probes), "staged": list(c.staged)}

    def count(self, per_vertex=None, total_dev=None, tuning: Optional[Tuning] = None,
              stream=None, sync: bool = True):
        """tc_count.  ``per_vertex``: None, True (allocate) or a CUDA uint64
        tensor of n entries (int64 accepted).  ``total_dev``: optional CUDA
        uint64/int64 tensor of one entry.  Returns the total (int) when sync,
        else None; with per_vertex=True also returns the tensor."""
        import torch
        pv = per_vertex
        if pv is True:
            pv = torch.empty(max(self.n, 1), dtype=torch.int64, device="cuda")
        total = ctypes.c_uint64(0)
        st = _stream_ptr(stream)
        _check(load().tc_count(self._h, ctypes.byref(tuning) if tuning is not None else None,
                               ctypes.addressof(total) if sync else None,
                               total_dev.data_ptr() if total_dev is not None else None,
                               pv.data_ptr() if pv is not None else None, st))
        t = int(total.value) if sync else None
        if per_vertex is True:
            return t, pv[: self.n]
        return t


    def offload(self, stream=None) -> None:
        """tc_graph_offload: move the count's arrays to page-locked host
        memory and free the device arena (then only count_tiled counts it)."""
        _check(load().tc_graph_offload(self._h, _stream_ptr(stream)))

    def count_tiled(self, budget_bytes: int, per_vertex: bool = False,
                    allocator: Optional[Allocator] = None, tuning: Optional[Tuning] = None,
                    stream=None):
        """tc_count_tiled: count an offloaded graph within budget_bytes of
        device memory.  Returns (total, per-vertex uint64 numpy or None,
        tiling stats)."""
        total = ctypes.c_uint64(0)
        pv = np.zeros(max(self.n, 1), dtype=np.uint64) if per_vertex else None
        ts = TiledStats()
        _check(load().tc_count_tiled(self._h, int(budget_bytes),
                                     ctypes.byref(allocator) if allocator is not None else None,
                                     ctypes.byref(tuning) if tuning is not None else None,
                                     ctypes.addressof(total), pv.ctypes.data if pv is not None else None,
                                     ctypes.byref(ts), _stream_ptr(stream)))
        return (int(total.value), pv[: self.n] if pv is not None else None,
                {f: int(getattr(ts, f)) for f, _ in TiledStats._fields_})


class Batch:
    """tc_batch_*: many graphs counted by one persistent launch (replayed
    from a captured CUDA graph).  The graphs must outlive the batch."""

    def __init__(self, graphs, tuning: Optional[Tuning] = None):
        self.graphs = list(graphs)
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.handle for g in self.graphs])
        h = ctypes.c_void_p(0)
        _check(load().tc_batch_create(arr, len(self.graphs),
                                      ctypes.byref(tuning) if tuning is not None else None,
                                      None, ctypes.byref(h)))
        self._h = h

    def count(self, totals=None, stream=None):
        """Counts every graph; returns (and fills) a CUDA int64 tensor of totals."""
        import torch
        if totals is None:
            totals = torch.empty(len(self.graphs), dtype=torch.int64, device="cuda")
        _check(load().tc_batch_count(self._h, totals.data_ptr(), _stream_ptr(stream)))
        return totals

    def autotune(self, reps: int = 3, stream=None) -> Tuning:
        t = Tuning()
        _check(load().tc_batch_autotune(self._h, reps, ctypes.byref(t), _stream_ptr(stream)))
        return t

    def count_stats(self, stream=None) -> dict:
        c = CountStats()
        _check(load().tc_batch_get_count_stats(self._h, ctypes.byref(c), _stream_ptr(stream)))
        return {"triangles": int(c.triangles), "units": list(c.units), "tasks": list(c.tasks),
                "probes": list(c.probes), "staged": list(c.staged)}

    def free(self) -> None:
        if self._h.value:
            load().tc_batch_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """tc_server_*: continuously batched counting of seeded RMAT requests."""

    def __init__(self, hbm_budget_bytes: int = 0, workers: int = 0, max_batch: int = 0,
                 max_tick_pairs: int = 0, device: int = -1):
        cfg = ServerConfig(hbm_budget_bytes, workers, max_batch, max_tick_pairs, device, 0)
        h = ctypes.c_void_p(0)
        _check(load().tc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._buf = (ServerResult * 4096)()

    def now(self) -> float:
        return float(load().tc_server_now(self._h))

    def submit_rmat(self, seed: int, scale: int, n: int, num_pairs: int,
                    thresholds: Optional[tuple] = None, t_arrival: Optional[float] = None) -> int:
        """Queue one request; returns its ticket (raises TCError on TC_EBUSY/EINVAL)."""
        if thresholds is None:
            from .inputs import rmat_thresholds
            thresholds = rmat_thresholds()
        spec = RmatSpec(seed & (2**64 - 1), scale, 0, n, num_pairs, *thresholds, 0)
        t = ctypes.c_int64(-1)
        _check(load().tc_server_submit_rmat(self._h, ctypes.byref(spec),
                                            self.now() if t_arrival is None else t_arrival,
                                            ctypes.byref(t)))
        return int(t.value)

    def submit_many(self, specs, thresholds: Optional[tuple] = None,
                    t_arrival: Optional[list] = None) -> list:
        """Queue several requests at once (tc_server_submit_rmat_many): specs
        are (seed, scale, n, num_pairs) tuples; returns their tickets."""
        if thresholds is None:
            from .inputs import rmat_thresholds
            thresholds = rmat_thresholds()
        k = len(specs)
        arr = (RmatSpec * max(k, 1))()
        for i, (seed, scale, n, num_pairs) in enumerate(specs):
            arr[i] = RmatSpec(seed & (2**64 - 1), scale, 0, n, num_pairs, *thresholds, 0)
        now = self.now()
        ta = (ctypes.c_double * max(k, 1))(*(t_arrival if t_arrival is not None else [now] * k))
        tk = (ctypes.c_int64 * max(k, 1))()
        _check(load().tc_server_submit_rmat_many(self._h, arr, k, ta, tk))
        return [int(tk[i]) for i in range(k)]

    def poll(self, wait_ms: int = 0) -> list:
        """Finished results as dicts (ticket, triangles, times, status, tick
        size, the tick's device span)."""
        cnt = ctypes.c_int32(0)
        out = []
        while True:
            _check(load().tc_server_poll(self._h, self._buf, len(self._buf), ctypes.byref(cnt),
                                         wait_ms if not out else 0))
            for i in range(cnt.value):
                r = self._buf[i]
                out.append({"ticket": int(r.ticket), "triangles": int(r.triangles),
                            "t_arrival": r.t_arrival, "t_admit": r.t_admit, "t_done": r.t_done,
                            "status": int(r.status), "tick_requests": int(r.tick_requests),
                            "tick_pairs": int(r.tick_pairs), "t_dev_start": r.t_dev_start,
                            "t_dev_end": r.t_dev_end})
            if cnt.value < len(self._buf):
                return out

    def drain(self, timeout_ms: int = 600000) -> None:
        _check(load().tc_server_drain(self._h, timeout_ms))

    def stats(self) -> dict:
        s = ServerStats()
        _check(load().tc_server_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def free(self) -> None:
        if self._h.value:
            load().tc_server_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def count_batch(graphs, tuning: Optional[Tuning] = None, stream=None):
    """tc_count_batch: one-shot batched count; returns a CUDA int64 tensor."""
    import torch
    graphs = list(graphs)
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle for g in graphs])
    totals = torch.empty(len(graphs), dtype=torch.int64, device="cuda")
    _check(load().tc_count_batch(arr, len(graphs),
                                 ctypes.byref(tuning) if tuning is not None else None,
                                 totals.data_ptr(), _stream_ptr(stream)))
    return totals


def preprocess(src, dst, n: int, offsets: Optional[int] = None, stream=None,
               allocator: Optional[Allocator] = None) -> Graph:
    """tc_preprocess.  src/dst: int32 CUDA tensors (device input) or int32
    numpy arrays / CPU tensors (host input, copied by the library)."""
    ps, dev_s = _ptr(src)
    pd, dev_d = _ptr(dst)
    assert dev_s == dev_d, "src and dst must live on the same side"
    num = int(src.shape[0])
    assert int(dst.shape[0]) == num
    flags = TC_INPUT_ON_DEVICE if dev_s else 0
    if offsets == 32:
        flags |= TC_OFFSETS_32
    elif offsets == 64:
        flags |= TC_OFFSETS_64
    h = ctypes.c_void_p(0)
    _check(load().tc_preprocess(ps, pd, num, n, flags,
                                ctypes.byref(allocator) if allocator is not None else None,
                                _stream_ptr(stream), ctypes.byref(h)))
    return Graph(h.value, n)


def preprocess_components(src, dst, vertex_prefix, offsets: Optional[int] = None,
                          stream=None) -> Graph:
    """tc_preprocess_components: the disjoint union of graphs whose vertex
    ranges are given by ``vertex_prefix`` (num_comps + 1 ints, starting at 0)."""
    ps, dev_s = _ptr(src)
    pd, dev_d = _ptr(dst)
    assert dev_s == dev_d
    vp_ = np.ascontiguousarray(np.asarray(vertex_prefix, dtype=np.int64))
    flags = TC_INPUT_ON_DEVICE if dev_s else 0
    if offsets == 32:
        flags |= TC_OFFSETS_32
    elif offsets == 64:
        flags |= TC_OFFSETS_64
    h = ctypes.c_void_p(0)
    _check(load().tc_preprocess_components(ps, pd, int(src.shape[0]), vp_.ctypes.data,
                                           vp_.size - 1, flags, None, _stream_ptr(stream),
                                           ctypes.byref(h)))
    g = Graph(h.value, int(vp_[-1]))
    g.num_comps = vp_.size - 1
    return g


def count_components(g: Graph, tuning: Optional[Tuning] = None, out=None, stream=None):
    """tc_count_components: per-component totals as a CUDA int64 tensor."""
    import torch
    if out is None:
        out = torch.empty(g.num_comps, dtype=torch.int64, device="cuda")
    _check(load().tc_count_components(g._h, ctypes.byref(tuning) if tuning is not None else None,
                                      out.data_ptr(), _stream_ptr(stream)))
    return out


def triangles(src: np.ndarray, dst: np.ndarray, n: int, per_vertex: bool = False,
              offsets: Optional[int] = None, stream=None, out: Optional[np.ndarray] = None):
    """tc_triangles on host arrays; returns total (and per-vertex numpy,
    written into ``out`` -- n uint64, e.g. a pinned buffer -- when given)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    total = ctypes.c_uint64(0)
    pv = None
    if per_vertex:
        pv = out if out is not None else np.zeros(max(n, 1), dtype=np.uint64)
        assert pv.dtype in (np.uint64, np.int64) and pv.flags["C_CONTIGUOUS"] and pv.size >= n
    flags = {None: 0, 32: TC_OFFSETS_32, 64: TC_OFFSETS_64}[offsets]
    _check(load().tc_triangles(src.ctypes.data, dst.ctypes.data, src.shape[0], n, flags,
                               _stream_ptr(stream), ctypes.addressof(total),
                               pv.ctypes.data if pv is not None else None))
    if per_vertex:
        return int(total.value), pv[:n]
    return int(total.value)


def triangles_timing() -> dict:
    """tc_triangles_get_timing: the phase split of this thread's last
    tc_triangles call (device phases from CUDA events, wall time on the host)."""
    t = TrianglesTiming()
    _check(load().tc_triangles_get_timing(ctypes.byref(t)))
    out = {f: float(getattr(t, f)) for f, _ in TrianglesTiming._fields_[:6]}
    out["input_pinned"] = bool(t.input_pinned)
    out["upload_method"] = {1: "copy engine", 2: "SM loads"}.get(int(t.upload_method), "none")
    out["ce_slice_gbs"] = float(t.ce_slice_gbs)
    out["sm_slice_gbs"] = float(t.sm_slice_gbs)
    return out


def triangles_static(src, dst, n: int, per_vertex=None, stream=None) -> int:
    """tc_triangles_static: count a small graph whose pairs are CUDA int32
    tensors without any device allocation by the library (buffers come from
    its fixed static scratch; see include/tc.h for the limits and the rules
    on overlapping calls).  ``per_vertex``: None or a CUDA int64 tensor of n
    entries that receives the per-vertex counts.  Returns the total."""
    import torch
    ps, dev_s = _ptr(src)
    pd, dev_d = _ptr(dst)
    assert dev_s and dev_d, "tc_triangles_static takes device pairs"
    assert int(dst.shape[0]) == int(src.shape[0]), "src and dst differ in length"
    dev = src.device
    if per_vertex is not None:
        assert (isinstance(per_vertex, torch.Tensor) and per_vertex.is_cuda
                and per_vertex.device == dev), "per_vertex must be a CUDA tensor on src's device"
        assert per_vertex.dtype in (torch.int64, torch.uint64), "per_vertex must be 64-bit"
        assert per_vertex.is_contiguous() and per_vertex.numel() >= n, "per_vertex needs n entries"
    # The library works on `lib_stream`; torch allocates `total` (and the
    # caller made the inputs) on its current stream.  The library stream waits
    # for the current one before the call, and the current one waits for the
    # library stream before the total is read back.
    cur = torch.cuda.current_stream(dev)
    st = _stream_ptr(stream)
    lib_stream = cur if st == cur.cuda_stream else (
        stream if isinstance(stream, torch.cuda.Stream)
        else torch.cuda.ExternalStream(st, device=dev))
    total = torch.empty(1, dtype=torch.int64, device=dev)
    if lib_stream is not cur:
        lib_stream.wait_stream(cur)
    _check(load().tc_triangles_static(ps, pd, int(src.shape[0]), n, total.data_ptr(),
                                      per_vertex.data_ptr() if per_vertex is not None else None,
                                      st))
    if lib_stream is not cur:
        cur.wait_stream(lib_stream)
    return int(total.item())


def generate_rmat(seed: int, scale: int, num_pairs: int, n: Optional[int] = None, e0: int = 0,
                  thresholds: Optional[tuple[int, int, int]] = None, out=None, stream=None):
    """tc_generate_rmat into (src, dst) int32 CUDA tensors (allocated if out is None)."""
    import torch
    if n is None:
        n = 1 << scale
    if thresholds is None:
        from .inputs import rmat_thresholds
        thresholds = rmat_thresholds()
    if out is None:
        src = torch.empty(num_pairs, dtype=torch.int32, device="cuda")
        dst = torch.empty(num_pairs, dtype=torch.int32, device="cuda")
    else:
        src, dst = out
    t1, t2, t3 = thresholds
    _check(load().tc_generate_rmat(seed & (2**64 - 1), scale, n, e0, num_pairs, t1, t2, t3,
                                   src.data_ptr(), dst.data_ptr(), _stream_ptr(stream)))
    return src, dst
