#!/usr/bin/env python
"""Benchmark: exact triangle counting on one GB300 per rank.

One step is the whole hot path on one synthetic graph already resident in
HBM: tc_preprocess (simple-graph conversion, degree-order relabel, U CSR,
task lists, units) followed by tc_count (total, and per-vertex counts where
the workload asks for them).  The metric is undirected edges per second:
m (simple undirected edges, nnz(U)) / step time, summed over ranks.

Workloads (seeded, synthetic, shaped like the paper's graph500 RMAT graphs,
with a Chung-Lu power-law graph standing in for its skewed social graphs):
  rmat-s26   RMAT scale 26, edge factor 16, a/b/c/d .57/.19/.19/.05,
             int64 offsets, total + per-vertex counts          (default)
  rmat-s14   RMAT scale 14, edge factor 16, int32 offsets, total only
  chunglu    Chung-Lu, n = 50M, exponent 2.1, mean degree 40,
             expected degrees capped at 1M, int64 offsets, total only

Multi-GPU: replicas only (each rank counts its own graph, seed + rank; no
collective on the data path).  Printed: one JSON line from rank 0.

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload: a smaller RMAT graph of the same family.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "rmat-s26": dict(kind="rmat", scale=26, edge_factor=16, offsets=64, per_vertex=True,
                     desc="RMAT scale 26 (67,108,864 vertices), edge factor 16 "
                          "(1,073,741,824 generated pairs), a/b/c/d=0.57/0.19/0.19/0.05; "
                          "int64 offsets; total + per-vertex uint64 counts"),
    "rmat-s14": dict(kind="rmat", scale=14, edge_factor=16, offsets=32, per_vertex=False,
                     desc="RMAT scale 14 (16,384 vertices), edge factor 16 (262,144 generated "
                          "pairs), a/b/c/d=0.57/0.19/0.19/0.05; int32 offsets; total count"),
    "chunglu": dict(kind="chung_lu", n=50_000_000, gamma=2.1, mean_degree=40.0, wmax=1e6,
                    offsets=64, per_vertex=False,
                    desc="Chung-Lu power law, 50,000,000 vertices, exponent 2.1, mean expected "
                         "degree 40 (10^9 pairs), expected degree capped at 10^6; int64 offsets; "
                         "total count"),
    "serve": dict(kind="serve", rate=2000.0, seconds=60.0,
                  desc="open-loop Poisson arrivals at 2,000 requests/s for 60 s; request r is a "
                       "seeded RMAT graph with M = floor(2^(10+12U)) pairs (2^10..2^22), edge "
                       "factor uniform in 8..32, n = ceil(M/e), ids >= n redrawn; expanded on "
                       "the device; exact count per request"),
    "tiled": dict(kind="tiled", scale=24, edge_factor=16, budget_fraction=8, per_vertex=True,
                  desc="RMAT scale 24 (16,777,216 vertices), edge factor 16, int64 offsets, total + "
                       "per-vertex counts; the graph offloaded to host memory and counted within 1/8 "
                       "of its device arena, (row block, pivot block) tiles streamed through device "
                       "memory, against the same graph counted in device memory"),
    "batch4096": dict(kind="batch", graphs=4096, offsets=32, per_vertex=False,
                      desc="4096 independent graphs, even ids G(n,p), odd ids RMAT "
                           "(a/b/c/d=0.57/0.19/0.19/0.05, ids >= n redrawn), n = floor(2^(8+8U)), "
                           "mean degree 4+60U; int32 ids and offsets; one uint64 count per graph; "
                           "autotuned unit knobs"),
}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat-s26")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-scale", type=int, default=19,
                    help="RMAT scale of the oracle's bounded sample")
    ap.add_argument("--scale", type=int, default=None,
                    help="override the RMAT scale of the workload (small profiling cases)")
    ap.add_argument("--no-per-vertex", action="store_true",
                    help="count totals only (profiling the totals kernel; not the workload's metric)")
    ap.add_argument("--graphs", type=int, default=None,
                    help="override the number of graphs of the batch workload")
    ap.add_argument("--serve-rate", type=float, default=None, help="requests/s (serve workload)")
    ap.add_argument("--serve-seconds", type=float, default=None, help="arrival window (serve)")
    ap.add_argument("--serve-workers", type=int, default=3)
    return ap.parse_args()


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

def reduce_over_ranks(maxes, sums, device="cuda"):
    """Job-wide figures from per-rank ones: the max over ranks of each entry
    of `maxes` (times) and the sum of each entry of `sums` (work done).  The
    identity on a single rank (no process group)."""
    import torch
    import torch.distributed as dist
    mx = torch.tensor([float(x) for x in maxes], dtype=torch.float64, device=device)
    sm = torch.tensor([float(x) for x in sums], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if mx.numel():
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        if sm.numel():
            dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return [float(x) for x in mx], [float(x) for x in sm]


def gather_over_ranks(arr):
    """The concatenation over ranks (in rank order) of a 1-D numpy array."""
    import numpy as np
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1):
        return arr
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, arr)
    return np.concatenate([np.asarray(p) for p in parts])


# the headline metric of each workload kind, shared by both arms
METRICS = {
    "rmat": ("undirected edges/sec (exact triangle count: preprocess + count per step)", "edges/s"),
    "chung_lu": ("undirected edges/sec (exact triangle count: preprocess + count per step)", "edges/s"),
    "batch": ("undirected edges/sec (exact triangle count, 4096-graph batch, count step)", "edges/s"),
    "serve": ("served exact triangle counts: throughput with p50/p99 latency", "requests/s"),
    "tiled": ("undirected edges/sec (exact triangle count within a device budget, count step)", "edges/s"),
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _cpulist(text: str) -> set:
    cpus = set()
    for part in text.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def bind_near_gpu(dev: int) -> str:
    """Restrict this thread to the CPUs the system lists as local to the GPU
    (sysfs local_cpulist of its PCI function), so that page-locked buffers it
    allocates land in the memory next to the GPU.  Returns what was done."""
    import torch
    try:
        p = torch.cuda.get_device_properties(dev)
        bdf = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        text = open(f"/sys/bus/pci/devices/{bdf}/local_cpulist").read()
        cpus = _cpulist(text) & os.sched_getaffinity(0)
        if not cpus:
            return f"not bound: no allowed CPU in {bdf} local_cpulist {text.strip()}"
        os.sched_setaffinity(0, cpus)
        return f"bound to {bdf} local_cpulist {text.strip()} ({len(cpus)} CPUs)"
    except (OSError, AttributeError, ValueError) as e:
        return f"not bound: {e}"


def peaks() -> tuple[float, str]:
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s"


KERNEL_SOURCES = {"k_count": ("count.cu", "common.cuh", "tc_internal.cuh")}


def source_digest(kernel: str = "k_count") -> str:
    """Digest of the source files a kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1907_09575_gb300", "csrc")
    for name in KERNEL_SOURCES.get(kernel, ()):
        h.update(name.encode())
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, workload: str, units: float, per_vertex: bool = True):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled
    by units processed when the capture was a smaller case; None when absent,
    when the kernel sources changed since the capture, or when the capture was
    of the other instance (per-vertex or totals only)."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None, "no ncu capture committed"
    e = rec.get(kernel)
    if not e or e.get("source_digest") != source_digest(kernel):
        return None, "kernel changed since the ncu capture" if e else "no capture of this kernel"
    key = "per_vertex" if per_vertex else "totals"
    c = e.get(key)
    if not c:
        return None, f"no capture of the {key} instance"
    if not c.get("scales_with_units", False):
        return None, (f"ncu capture of {c['case']}: {c['dram_bytes'] / 1e9:.1f} GB of DRAM traffic against "
                      f"{c['alg_bytes'] / 1e9:.1f} GB algorithmic ({c['note']}); it does not scale to a "
                      f"full launch by {c['unit_name']}, and the full-size counter capture is not repeated")
    per_unit = c["dram_bytes"] / max(c["units"], 1)
    return per_unit * units, f"ncu capture of {c['case']} scaled by units ({c['unit_name']})"


def alg_bytes_count(kstats: dict, off_bytes: int) -> float:
    """Algorithmic bytes of one count kernel launch (warp and CTA units): per
    unit its record (32 B) and the pivot row bounds (2 offsets); per staged
    pivot entry 4 B; per task its record (16 B); per probe the 4-B entry of
    U_i read.  Per-vertex flushes are not counted (atomics)."""
    return (sum(kstats["units"]) * (32 + 2 * off_bytes) + 4 * sum(kstats["staged"])
            + 16 * sum(kstats["tasks"]) + 4 * sum(kstats["probes"]))


# ----------------------------------------------------------------------------
# reference arm: the CPU oracle on a bounded sample
# ----------------------------------------------------------------------------

def run_reference(args, wl):
    """The CPU oracle (single thread) on a bounded sample of the same
    workload, each step a few seconds of work, same metric and unit."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1907_09575_gb300 import inputs
    oracle.build()
    kind = wl["kind"]
    metric, unit = METRICS[kind]
    if kind == "rmat":
        scale = min(wl["scale"], args.cpu_sample_scale)   # the sample cpu_baseline times
        specs = [inputs.rmat_graph(args.seed, scale, wl["edge_factor"])]
        sample = (f"RMAT scale {scale}, edge factor {wl['edge_factor']} per step"
                  + (" (the whole workload)" if scale == wl["scale"] else ""))
    elif kind == "chung_lu":
        specs = [inputs.chung_lu_graph(args.seed, n=1_000_000, gamma=wl["gamma"],
                                       mean_degree=wl["mean_degree"], wmax=wl["wmax"])]
        sample = "Chung-Lu with the same law on 1,000,000 vertices per step"
    elif kind == "batch":
        specs = [inputs.batch_member(args.seed, k) for k in range(64)]
        sample = "the first 64 graphs of the batch per step"
    elif kind == "tiled":
        scale = min(wl["scale"], args.cpu_sample_scale)
        specs = [inputs.rmat_graph(args.seed, scale, wl["edge_factor"])]
        sample = f"RMAT scale {scale}, edge factor {wl['edge_factor']} per step"
    else:
        specs = [inputs.serve_request(args.seed, r) for r in range(24)]
        sample = "the first 24 requests of the stream per step, counted one after another"
    data = [(sp, sp.generate()) for sp in specs]
    times, work = [], 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        w = 0
        for sp, (src, dst) in data:
            total, st = oracle.count(src, dst, sp.n, stats=True)
            w += st["m"] if unit == "edges/s" else 1
        dt = time.perf_counter() - t0
        work = w
        if it >= args.warmup:
            times.append(dt)
    step_s = sum(times) / len(times)
    value = work / step_s
    sample += f" ({work} {'edges' if unit == 'edges/s' else 'requests'}); oracle preprocess+count, single thread"
    line = {
        "impl": "reference", "metric": metric,
        "value": value, "unit": unit, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"], "seed": args.seed,
                   "sample": sample, "parallelism": "one host core (rank 0)"},
        "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def make_inputs(wl, seed, torch, tc, inputs):
    if wl["kind"] == "rmat":
        n = 1 << wl["scale"]
        num = wl["edge_factor"] * n
        s, d = tc.generate_rmat(seed, wl["scale"], num)
        return s, d, n, num, "device-generated seeded RMAT"
    spec = inputs.chung_lu_graph(seed, wl["n"], wl["gamma"], wl["mean_degree"], wl["wmax"])
    hs, hd = spec.generate()
    return (torch.from_numpy(hs).cuda(), torch.from_numpy(hd).cuda(), spec.n, spec.num_pairs,
            "host-generated seeded Chung-Lu, uploaded before timing")


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def cpu_baseline(args, per_vertex):
    """The oracle (one thread) and the OpenMP counter (all host cores) on the
    same bounded sample: RMAT scale cpu_sample_scale of the workload's family
    (the sample the reference arm times too)."""
    import cpu_parallel
    import oracle
    from paper_1907_09575_gb300 import inputs
    oracle.build()
    cpu_parallel.build()
    spec = inputs.rmat_graph(args.seed, args.cpu_sample_scale, 16)
    src, dst = spec.generate()
    t0 = time.perf_counter()
    total, st = oracle.count(src, dst, spec.n, stats=True)
    dt = time.perf_counter() - t0
    sample = (f"RMAT scale {args.cpu_sample_scale}, edge factor 16 ({spec.num_pairs} pairs, "
              f"m={st['m']}, {total} triangles)")
    base = {"value": st["m"] / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample}: the oracle's preprocess+count, single thread, {dt:.1f} s",
            "seconds": dt}
    cpu_parallel.count(src, dst, spec.n, per_vertex=per_vertex)           # warm (threads, pages)
    t0 = time.perf_counter()
    ptotal, _, pst = cpu_parallel.count(src, dst, spec.n, per_vertex=per_vertex)
    pdt = time.perf_counter() - t0
    assert ptotal == total, (ptotal, total)
    par = {"value": pst["m"] / pdt, "unit": "edges/s", "cores": pst["threads"],
           "nproc": os.cpu_count(), "cpu_model": cpu_model(),
           "kind": "OpenMP shared-memory <j,i,k> map-based counter (cpu_parallel/)",
           "sample": f"{sample}: preprocess+count" + (" with per-vertex counts" if per_vertex else "")
                     + f", {pst['threads']} threads, {pdt:.2f} s; total equals the oracle's",
           "seconds": pdt}
    return base, par


def run_ours(args, wl):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1907_09575_gb300 import inputs, tc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tc.load()
    seed = args.seed + rank
    src, dst, n, num_pairs, data = make_inputs(wl, seed, torch, tc, inputs)
    pv = torch.empty(max(n, 1), dtype=torch.int64, device="cuda") if wl["per_vertex"] else None
    tdev = torch.zeros(1, dtype=torch.int64, device="cuda")
    off = wl["offsets"]

    def step():
        g = tc.preprocess(src, dst, n, offsets=off)
        g.count(per_vertex=pv, total_dev=tdev, sync=False)
        return g

    def barrier():
        if ws > 1:
            dist.barrier()

    facts = None
    for _ in range(args.warmup):
        g = step()
        facts = g.stats()
        g.free()
    torch.cuda.synchronize()
    g = step()
    facts = g.stats()
    total = int(tdev.item())
    g.free()

    # --- timed region: K whole steps -------------------------------------
    # Per-launch event timing adds host work to every launch; a step of a
    # few dozen launches under 20 ms is timed without it and its kernels are
    # timed in a second loop of the same steps.
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    g = step()
    g.free()
    ev1.record()
    torch.cuda.synchronize()
    profile_in_loop = ev0.elapsed_time(ev1) >= 20.0
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    tc.profile_enable(profile_in_loop)
    l0 = tc.kernel_launches()
    ev0.record()
    for _ in range(args.steps):
        g = step()
        g.free()
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    launches = tc.kernel_launches() - l0
    prof = tc.profile_read() if profile_in_loop else None
    tc.profile_enable(False)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    if not profile_in_loop:
        tc.profile_enable(True)
        for _ in range(args.steps):
            g = step()
            g.free()
        torch.cuda.synchronize()
        prof = tc.profile_read()
        tc.profile_enable(False)
    (ms,), (m_all,) = reduce_over_ranks([ms], [facts["m"]])
    value = m_all / (ms / 1e3)

    # --- count alone (the paper's "tct"), CSR resident -------------------
    g = tc.preprocess(src, dst, n, offsets=off)
    for _ in range(2):
        g.count(per_vertex=pv, total_dev=tdev, sync=False)
    torch.cuda.synchronize()
    tc.profile_enable(True)
    ev0.record()
    for _ in range(args.steps):
        g.count(per_vertex=pv, total_dev=tdev, sync=False)
    ev1.record()
    torch.cuda.synchronize()
    cprof = tc.profile_read()
    tc.profile_enable(False)
    count_ms = ev0.elapsed_time(ev1) / args.steps
    kst = g.count_stats()
    g.free()

    # --- roofline of the dominant kernel of the step ---------------------
    hbm, peak_src = peaks()
    step_kernel_ms = sum(v[1] for v in prof.values())
    top = max(prof.items(), key=lambda kv: kv[1][1])
    kname, (klaunch, kms) = top
    roof = None
    if kname == "k_count":
        b_launch = alg_bytes_count(kst, facts["offset_bytes"])
        avg_ms = kms / klaunch
        achieved = b_launch / (avg_ms / 1e3) / 1e9
        traffic, tnote = traffic_for(kname, args.workload, sum(kst["probes"]), wl["per_vertex"])
        roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                "traffic_note": tnote, "peak_source": peak_src,
                "alg_bytes_per_launch": b_launch, "avg_launch_ms": avg_ms,
                "share_of_step_kernel_time": kms / step_kernel_ms,
                "probes_per_launch": sum(kst["probes"])}
    else:
        roof = {"kernel": kname, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s",
                "frac": None, "traffic": None, "peak_source": peak_src,
                "share_of_step_kernel_time": kms / step_kernel_ms,
                "note": "dominant kernel is a preprocessing kernel"}

    # --- end to end through the one-shot C ABI call, host buffers ------------
    e2e = None
    if not args.no_e2e:
        affinity = os.sched_getaffinity(0)
        numa_note = bind_near_gpu(local)
        hs = torch.empty(num_pairs, dtype=torch.int32, pin_memory=True)
        hd = torch.empty(num_pairs, dtype=torch.int32, pin_memory=True)
        hs.copy_(src)
        hd.copy_(dst)
        hpv = torch.empty(max(n, 1), dtype=torch.int64, pin_memory=True) if wl["per_vertex"] else None
        hs_np, hd_np = hs.numpy(), hd.numpy()
        hpv_np = hpv.numpy() if hpv is not None else None
        tc.triangles(hs_np, hd_np, n, per_vertex=wl["per_vertex"], offsets=off, out=hpv_np)
        torch.cuda.synchronize()
        # the box's own pinned-upload rate of the same buffer, for comparison
        up = torch.empty(num_pairs, dtype=torch.int32, device="cuda")
        up.copy_(hs, non_blocking=True)
        torch.cuda.synchronize()
        ev0.record()
        up.copy_(hs, non_blocking=True)
        ev1.record()
        torch.cuda.synchronize()
        torch_h2d_gbs = 4 * num_pairs / (ev0.elapsed_time(ev1) / 1e3) / 1e9
        del up
        barrier()
        t0 = time.perf_counter()
        splits = []
        for _ in range(args.steps):
            r = tc.triangles(hs_np, hd_np, n, per_vertex=wl["per_vertex"], offsets=off, out=hpv_np)
            splits.append(tc.triangles_timing())
        torch.cuda.synchronize()
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.steps
        (e2e_s,), _ = reduce_over_ranks([e2e_s], [])
        e2e_total = r[0] if isinstance(r, tuple) else r
        assert e2e_total == total, (e2e_total, total)
        split = {k: (sum(x[k] for x in splits) / len(splits) if isinstance(splits[0][k], float)
                     else splits[-1][k]) for k in splits[0]}
        e2e = {"value": m_all / e2e_s, "unit": "edges/s", "ms_per_step": e2e_s * 1e3,
               "h2d_bytes_per_step": 8 * num_pairs,
               "d2h_bytes_per_step": 8 + (8 * n if wl["per_vertex"] else 0),
               "call": "tc_triangles (host pairs in pinned memory -> host total"
                       + (" + per-vertex)" if wl["per_vertex"] else ")"),
               "split_ms": {k: (round(v, 3) if isinstance(v, float) else v) for k, v in split.items()},
               "torch_pinned_h2d_gbs": torch_h2d_gbs, "host_buffers": numa_note}
        del hs, hd, hpv
        os.sched_setaffinity(0, affinity)

    cpu = cpu_par = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, cpu_par = cpu_baseline(args, wl["per_vertex"])

    if ws > 1:
        dist.barrier()
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    top_kernels = sorted(prof.items(), key=lambda kv: -kv[1][1])[:8]
    line = {
        "metric": METRICS[wl["kind"]][0],
        "value": value, "unit": "edges/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32 ids / uint64 counts",
        "data": f"synthetic ({data})",
        "config": {"workload": args.workload, "desc": wl["desc"], "n": n, "num_pairs": num_pairs,
                   "m": facts["m"], "offsets": facts["offset_bytes"] * 8,
                   "per_vertex": wl["per_vertex"], "seed": args.seed,
                   "l2": f"inputs larger than L2 ({8 * num_pairs / 1e9:.2f} GB of pairs per step)"
                         if 8 * num_pairs > 256e6 else
                         f"inputs ({8 * num_pairs / 1e6:.1f} MB) fit in L2: small-graph latency workload",
                   "kernel_timing": "events around every launch inside the timed loop" if profile_in_loop
                                    else "a second loop of the same steps (events would add host work "
                                         "to each of the step's short launches)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "triangles": total,
        "count_only": {"value": m_all / (count_ms / 1e3), "unit": "edges/s", "ms": count_ms,
                       "kernels": {k: [v[0], round(v[1], 3)] for k, v in cprof.items()}},
        "roofline": roof,
        "cpu_baseline": cpu,
        "cpu_parallel": cpu_par,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "graph": {k: facts[k] for k in ("m", "max_deg", "max_outdeg", "tasks", "probes",
                                        "small_units", "large_units", "device_bytes")},
        "count_work": kst,
        "step_kernels_ms": {k: [v[0], round(v[1], 3)] for k, v in top_kernels},
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# batched form: many graphs, one persistent launch
# ----------------------------------------------------------------------------

def run_batch(args, wl):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1907_09575_gb300 import inputs, tc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tc.load()
    ngraphs = args.graphs or wl["graphs"]
    seed = args.seed + rank
    t0 = time.perf_counter()
    graphs, pairs, ms_list = [], 0, []
    host_pairs = []   # for the end-to-end pass: all graphs as one disjoint union
    vprefix = [0]
    for k in range(ngraphs):
        spec = inputs.batch_member(seed, k)
        hs, hd = spec.generate()
        pairs += hs.size
        if not args.no_e2e:
            host_pairs.append((hs.astype(np.int64) + vprefix[-1], hd.astype(np.int64) + vprefix[-1]))
        vprefix.append(vprefix[-1] + spec.n)
        graphs.append(tc.preprocess(torch.from_numpy(hs).cuda(), torch.from_numpy(hd).cuda(),
                                    spec.n, offsets=wl["offsets"]))
    if not args.no_e2e:
        union_s = torch.from_numpy(np.concatenate([a for a, _ in host_pairs]).astype(np.int32)).pin_memory()
        union_d = torch.from_numpy(np.concatenate([b for _, b in host_pairs]).astype(np.int32)).pin_memory()
        host_pairs = None
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    facts = [g.stats() for g in graphs]
    m_all = float(sum(f["m"] for f in facts))

    b = tc.Batch(graphs)
    t0 = time.perf_counter()
    tuning = b.autotune(reps=2)
    tune_s = time.perf_counter() - t0
    totals = torch.zeros(ngraphs, dtype=torch.int64, device="cuda")

    def barrier():
        if ws > 1:
            dist.barrier()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        b.count(totals)
    torch.cuda.synchronize()
    want = totals.clone()
    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    tc.profile_enable(True)
    l0 = tc.kernel_launches()
    ev0.record()
    for _ in range(args.steps):
        b.count(totals)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    launches = tc.kernel_launches() - l0
    prof = tc.profile_read()
    tc.profile_enable(False)
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    kst = b.count_stats()
    assert torch.equal(totals, want)

    # the same kernel, one graph per launch, at the library's default tuning:
    # what a caller counting the graphs one by one gets (the batch's tuned
    # knobs suit many graphs in one launch, not one small graph at a time)
    per = torch.zeros(ngraphs, dtype=torch.int64, device="cuda")
    for _ in range(max(1, args.warmup)):
        for k, g in enumerate(graphs):
            g.count(total_dev=per[k:k + 1], sync=False)
    torch.cuda.synchronize()
    tc.profile_enable(True)
    ev0.record()
    for _ in range(args.steps):
        for k, g in enumerate(graphs):
            g.count(total_dev=per[k:k + 1], sync=False)
    ev1.record()
    torch.cuda.synchronize()
    pprof = tc.profile_read()
    tc.profile_enable(False)
    ms_one = ev0.elapsed_time(ev1) / args.steps
    assert torch.equal(per, totals), "one-per-launch totals differ from the batch"

    (ms, ms_one), (m_tot,) = reduce_over_ranks([ms, ms_one], [m_all])
    value = m_tot / (ms / 1e3)

    hbm, peak_src = peaks()
    kb = prof.get("k_count_batch", (args.steps, ms * args.steps))
    b_launch = alg_bytes_count(kst, wl["offsets"] // 8)
    achieved = b_launch / (kb[1] / kb[0] / 1e3) / 1e9
    roof = {"kernel": "k_count (batched, one captured launch)", "bound": "hbm",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "traffic_note": "no ncu capture of the batched launch committed",
            "peak_source": peak_src, "alg_bytes_per_launch": b_launch,
            "avg_launch_ms": kb[1] / kb[0]}

    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        us_np, ud_np = union_s.numpy(), union_d.numpy()
        for _ in range(args.steps):
            gu = tc.preprocess_components(us_np, ud_np, vprefix)
            host_totals = tc.count_components(gu).cpu()
            gu.free()
        e2e_s = (time.perf_counter() - t0) / args.steps
        assert torch.equal(host_totals.cuda(), totals)
        e2e = {"value": m_tot / e2e_s, "unit": "edges/s", "ms_per_step": e2e_s * 1e3,
               "h2d_bytes_per_step": 8 * pairs, "d2h_bytes_per_step": 8 * ngraphs,
               "call": "tc_preprocess_components on the pinned host pairs of all graphs (one "
                       "disjoint union), tc_count_components, totals to host"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        mm, k = 0, 0
        while time.perf_counter() - t0 < 10.0 and k < ngraphs:
            hs, hd = inputs.batch_member(seed, k).generate()
            tot, st = oracle.count(hs, hd, inputs.batch_member(seed, k).n, stats=True)
            assert tot == int(totals[k])
            mm += st["m"]
            k += 1
        dt = time.perf_counter() - t0
        cpu = {"value": mm / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {k} graphs of the batch (m={mm}), oracle preprocess+count, "
                         f"single thread, {dt:.1f} s (includes host generation)"}
    if ws > 1:
        dist.barrier()
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRICS["batch"][0],
        "value": value, "unit": "edges/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32 ids / uint64 counts",
        "data": "synthetic (host-generated seeded G(n,p) and RMAT graphs)",
        "config": {"workload": args.workload, "desc": wl["desc"], "graphs": ngraphs,
                   "pairs": pairs, "m": int(m_tot), "seed": args.seed,
                   "l2": f"inputs larger than L2 (CSRs and task lists of {ngraphs} graphs)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "triangles": int(totals.sum().item()),
        "one_per_launch": {"value": m_tot / (ms_one / 1e3), "unit": "edges/s", "ms": ms_one,
                           "launches_per_step": sum(v[0] for v in pprof.values()) // max(args.steps, 1),
                           "tuning": "library default"},
        "batch_speedup": ms_one / ms,
        "tuning": {f: getattr(tuning, f) for f in ("small_max_outdeg", "warp_unit_tasks",
                                                   "cta_unit_tasks", "cta_threads", "slice_max",
                                                   "merge_max_outdeg")},
        "autotune_s": tune_s, "setup_s": setup_s,
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "count_work": kst,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# graphs larger than the device budget: the tiled count
# ----------------------------------------------------------------------------

def run_tiled(args, wl):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1907_09575_gb300 import tc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tc.load()
    n = 1 << wl["scale"]
    s, d = tc.generate_rmat(args.seed + rank, wl["scale"], wl["edge_factor"] * n)
    g = tc.preprocess(s, d, n, offsets=64)
    del s, d
    facts = g.stats()
    arena = facts["device_bytes"]
    budget = arena // wl["budget_fraction"]
    pv = torch.empty(n, dtype=torch.int64, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        g.count(per_vertex=pv, sync=True)
    ev0.record()
    for _ in range(args.steps):
        total = g.count(per_vertex=pv, sync=True)
    ev1.record()
    torch.cuda.synchronize()
    hbm_ms = ev0.elapsed_time(ev1) / args.steps
    want_pv = pv.cpu().numpy().astype(np.uint64)
    g.offload()
    for _ in range(max(1, args.warmup - 2)):
        g.count_tiled(budget, per_vertex=True)
    sampler = ClockSampler(local)
    sampler.start()
    tc.profile_enable(True)
    l0 = tc.kernel_launches()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t_total, t_pv, ts = g.count_tiled(budget, per_vertex=True)
    tiled_s = (time.perf_counter() - t0) / args.steps
    launches = tc.kernel_launches() - l0
    prof = tc.profile_read()
    tc.profile_enable(False)
    clocks = sampler.stop()
    g.free()
    assert t_total == total and np.array_equal(t_pv, want_pv)
    (tiled_s,), (m_all,) = reduce_over_ranks([tiled_s], [facts["m"]])
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    kc = prof.get("k_count", (1, 0.0))
    line = {
        "metric": METRICS["tiled"][0], "value": m_all / tiled_s, "unit": "edges/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tiled_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32 ids / uint64 counts", "data": "synthetic (device-generated seeded RMAT)",
        "config": {"workload": args.workload, "desc": wl["desc"], "n": n, "m": facts["m"],
                   "arena_bytes": arena, "budget_bytes": budget,
                   "l2": "graph arrays (host memory) far larger than L2",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "triangles": total,
        "in_hbm": {"ms": hbm_ms, "value": m_all / (hbm_ms / 1e3), "unit": "edges/s"},
        "tile_overhead": tiled_s * 1e3 / hbm_ms,
        "tiling": ts, "upload_gbs": ts["h2d_bytes"] / tiled_s / 1e9,
        "count_kernel_ms_per_step": kc[1] / args.steps,
        "e2e": {"value": m_all / tiled_s, "unit": "edges/s", "h2d_bytes_per_step": ts["h2d_bytes"],
                "d2h_bytes_per_step": 8 * n + 8,
                "note": "the count from host-resident arrays to host results is the timed call"},
        "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# served form: an open-loop Poisson stream of requests
# ----------------------------------------------------------------------------

def run_serve(args, wl):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1907_09575_gb300 import inputs, tc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tc.load()
    rate = args.serve_rate or wl["rate"]
    seconds = args.serve_seconds or wl["seconds"]
    seed = args.seed + rank
    arrivals = inputs.serve_arrivals(seed, rate, seconds)
    specs = [inputs.serve_request(seed, r) for r in range(arrivals.size)]
    t1, t2, t3 = inputs.rmat_thresholds()
    srv = tc.Server(hbm_budget_bytes=64 << 30, workers=args.serve_workers, max_batch=4096,
                    max_tick_pairs=1 << 28)

    # warm-up: the first requests of another seed, untimed
    for r in range(min(200, 50 * max(args.warmup, 1))):
        w = inputs.serve_request(seed + 1000, r)
        srv.submit_rmat(w.seed, w.scale, w.n, w.num_pairs, (t1, t2, t3))
    srv.drain()
    srv.poll()

    def barrier():
        if ws > 1:
            dist.barrier()

    sampler = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    mem0 = tc.memory_stats(local, reset_high=True)
    sampler.start()
    tc.profile_enable(True)
    l0 = tc.kernel_launches()
    t0 = srv.now()
    tickets = {}
    results = []
    nxt = 0
    while nxt < len(specs):
        now = srv.now() - t0
        while nxt < len(specs) and arrivals[nxt] <= now:
            sp = specs[nxt]
            tk = srv.submit_rmat(sp.seed, sp.scale, sp.n, sp.num_pairs, (t1, t2, t3),
                                 t_arrival=t0 + float(arrivals[nxt]))
            tickets[tk] = nxt
            nxt += 1
        results.extend(srv.poll())
        time.sleep(0.0002)
    srv.drain(timeout_ms=900000)
    t_end = srv.now()
    results.extend(srv.poll())
    launches = tc.kernel_launches() - l0
    prof = tc.profile_read()
    tc.profile_enable(False)
    clocks = sampler.stop()
    st = srv.stats()
    mem = tc.memory_stats(local)
    srv.free()
    assert len(results) == len(specs) and all(r["status"] == 0 for r in results)
    lat = np.array([r["t_done"] - r["t_arrival"] for r in results])
    qwait = np.array([r["t_admit"] - r["t_arrival"] for r in results])
    span = t_end - t0
    pairs = float(sum(sp.num_pairs for sp in specs))

    # every result of a bounded sample against its stand-alone count, the
    # small ones also against the oracle
    rng = np.random.default_rng(seed)
    by_ticket = {r["ticket"]: r for r in results}
    sample = rng.choice(list(by_ticket), size=min(200, len(by_ticket)), replace=False)
    import oracle
    oracle.build()
    checked_oracle = 0
    for tk in sample:
        sp = specs[tickets[int(tk)]]
        s, d = tc.generate_rmat(sp.seed, sp.scale, sp.num_pairs, n=sp.n)
        g = tc.preprocess(s, d, sp.n)
        alone = g.count()
        g.free()
        assert alone == by_ticket[int(tk)]["triangles"], (tk, alone)
        if sp.num_pairs <= (1 << 15) and checked_oracle < 60:
            hs, hd = sp.generate()
            assert oracle.count(hs, hd, sp.n) == alone
            checked_oracle += 1

    # job-wide: requests and pairs summed over the replicas, the longest span,
    # percentiles over every rank's requests
    (span,), (n_done, pairs) = reduce_over_ranks([span], [len(results), pairs])
    lat = gather_over_ranks(lat)
    qwait = gather_over_ranks(qwait)
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRICS["serve"][0],
        "value": n_done / span, "unit": "requests/s", "n_gpus": ws, "steps": 1,
        "warmup": args.warmup, "ms_per_step": span * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32 ids / uint64 counts",
        "data": "synthetic (seeded RMAT request specs expanded on the device)",
        "config": {"workload": args.workload, "desc": wl["desc"], "rate_hz": rate,
                   "seconds": seconds, "requests": int(n_done), "pairs": int(pairs),
                   "workers": args.serve_workers, "hbm_budget_bytes": 64 << 30,
                   "l2": "each tick's pairs and CSRs exceed L2 except for the smallest ticks",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                       "p99": float(np.percentile(lat, 99) * 1e3),
                       "mean": float(lat.mean() * 1e3), "max": float(lat.max() * 1e3)},
        "queue_wait_ms": {"p50": float(np.percentile(qwait, 50) * 1e3),
                          "p99": float(np.percentile(qwait, 99) * 1e3)},
        "pairs_per_s": pairs / span, "offered_pairs_per_s": pairs / seconds,
        "server": st, "checked": {"standalone_gpu": int(len(sample)), "oracle": checked_oracle},
        "device_overlap_frac": st["device_overlap_s"] / max(st["device_busy_s"], 1e-9),
        "memory": {"pool_used_high_bytes": mem["used_high"] - mem0["used"],
                   "admission_estimate_peak_bytes": st["peak_bytes_in_flight"],
                   "budget_bytes": 64 << 30},
        "e2e": {"value": n_done / span, "unit": "requests/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(8 * n_done),
                "note": "requests are generator specs expanded on the device; only totals return"},
        "gpu_launches": launches, "clocks": clocks,
        "kernels_ms": {k: [v[0], round(v[1], 2)] for k, v in
                       sorted(prof.items(), key=lambda kv: -kv[1][1])[:8]},
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    wl = dict(WORKLOADS[args.workload])
    if args.scale is not None:
        assert wl["kind"] == "rmat", "--scale applies to the RMAT workloads"
        wl["scale"] = args.scale
        wl["desc"] = f"{wl['desc']} [scale overridden to {args.scale}]"
        args.workload = f"{args.workload}@scale{args.scale}"
    if args.no_per_vertex and "per_vertex" in wl:
        wl["per_vertex"] = False
        wl["desc"] = f"{wl['desc']} [totals only]"
        args.workload = f"{args.workload}@totals"
    if args.impl == "reference":
        run_reference(args, wl)
    elif wl["kind"] == "batch":
        run_batch(args, wl)
    elif wl["kind"] == "serve":
        run_serve(args, wl)
    elif wl["kind"] == "tiled":
        run_tiled(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
