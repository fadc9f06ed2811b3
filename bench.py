#!/usr/bin/env python
"""Kernel-mix throughput of the co-scheduled runtime on GB300.

Workload (default): the eight-tenant mix — 64 kernels submitted at once, 8 of
each type in a seeded order: FP32 GEMM 1024^3, CSR SpMV 2^20 rows (power-law
rows, mean 16 nnz), Black-Scholes 4 Mi options, int32 pointer chase over a
64 MiB random cycle (65,536 chasers x 256 hops), FP32 triad 64 Mi, 256-bin
histogram of 64 Mi Zipf(1.1) bytes, escape-time 2048^2 (max 256 iterations),
bitonic sort of 2^22 uint32. Inputs are seeded synthetic arrays resident in
HBM (about 10 GB per step, far larger than L2).

One step = the whole hot path for one batch: submit the 64 descriptors,
plan (CP table, device-side FindCoSchedule), run the persistent co-scheduler,
retire completions. The same batch is also run as plain launches on 32
streams (multi-stream) and on one stream (serial FIFO) for the speedups.

Prints one JSON line (rank 0). --impl reference times the CPU oracle instead.
Multi-GPU: replicas only (every rank runs its own batch; no data exchange).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "kernel-mix throughput (kernels/s) & makespan speedup vs multi-stream on 1 GB300; p99 latency"
BATCH_WORKLOAD = ("batch of 512 tenants, types uniform over the eight mix kernels, grids log-uniform in "
                  "[1, 4096] blocks, problem sizes scaled to the grid, one persistent launch")
WORKLOAD = ("8-tenant mix, 64 kernels (8 each of FP32 GEMM 1024^3, CSR SpMV 1Mi rows power-law mean 16, "
            "Black-Scholes 4Mi, pointer-chase 64MiB x 65536 chasers x 256 hops, triad 64Mi, hist256 64Mi "
            "Zipf(1.1), escape-time 2048^2 max 256, bitonic 2^22), seeded order")


# ---------------------------------------------------------------------- ranks

def max_over_ranks(x: float, world: int, device: str) -> float:
    """The slowest rank's value (the step time every rank waits for)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(kernels_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: kernels all ranks processed per second of the
    slowest rank's step (replicas: every rank runs its own batch)."""
    return world * kernels_per_rank / (ms_per_step / 1e3)


# ---------------------------------------------------------------------- inputs

def _gen_one(job):
    name, cs, ti, size = job
    from workloads import gen
    return gen.gen_tenant(name, cs, ti, **size)


def mix_jobs(seed: int = 2, copies: int = 8):
    import numpy as np
    from paper_1303_5164_gb300.tenants import MIX_TYPES, SIZES_MIX
    order = [t for t in MIX_TYPES for _ in range(copies)]
    np.random.default_rng(seed).shuffle(order)
    return [(nm, seed, i, SIZES_MIX[nm]) for i, nm in enumerate(order)]


def batch_sizes(name: str, g: int) -> dict:
    """Problem size of a tenant whose (main-stage) grid is g blocks."""
    if name == "gemm_f32":
        a = 1 << (g.bit_length() - 1) // 2
        return dict(M=64 * a, N=64 * -(-g // a), K=512)
    if name == "spmv_csr":
        return dict(nrows=32 * g)
    if name == "blackscholes":
        return dict(n=256 * g)
    if name == "pchase":
        return dict(N=max(1 << 16, 4096 * g), nchasers=256 * g, hops=256)
    if name == "triad":
        return dict(n=4096 * g)
    if name == "hist256":
        return dict(n=32768 * g)
    if name == "escape":
        return dict(width=256, height=g, max_iter=256)
    if name == "bitonic":
        return dict(log2n=12 + g.bit_length() - 1)
    raise ValueError(name)


def batch_jobs(seed: int = 3, n: int = 512):
    """512 tenants: types uniform over the eight, grids log-uniform in [1, 4096]."""
    import numpy as np
    from paper_1303_5164_gb300.tenants import MIX_TYPES
    rng = np.random.default_rng(seed)
    types = rng.integers(0, len(MIX_TYPES), n)
    grids = np.minimum(4096, np.floor(np.exp(rng.uniform(0.0, np.log(4097.0), n)))).astype(int)
    return [(MIX_TYPES[t], seed, i, batch_sizes(MIX_TYPES[t], int(g))) for i, (t, g) in enumerate(zip(types, grids))]


SERVE_WORKLOAD = ("serving: open-loop Poisson arrivals of the eight mix kernel types (equal mix), sizes of the "
                  "64-kernel mix scaled 0.25x-4x log-uniform (five power-of-two buckets), admission by "
                  "declared device-memory footprint (cap 150 GB) and in-flight slots (608 = SMs x 4)")
SERVE_SCALES = (0.25, 0.5, 1.0, 2.0, 4.0)
# log-uniform scale on [1/4, 4] rounded to the nearest power of two in log2
SERVE_P = (0.125, 0.25, 0.25, 0.25, 0.125)


def serve_size(name: str, s: float) -> dict:
    """Size of a mix kernel scaled by s (work and bytes proportional to s)."""
    from paper_1303_5164_gb300.tenants import SIZES_MIX
    z = dict(SIZES_MIX[name])
    if name == "gemm_f32":
        z["M"] = int(z["M"] * s)
    elif name == "spmv_csr":
        z["nrows"] = int(z["nrows"] * s)
    elif name in ("blackscholes", "triad", "hist256"):
        z["n"] = int(z["n"] * s)
    elif name == "pchase":
        z["nchasers"] = int(z["nchasers"] * s)
    elif name == "escape":
        z["height"] = int(z["height"] * s)
    elif name == "bitonic":
        z["log2n"] = z["log2n"] + int(round(__import__("math").log2(s)))
    return z


def serve_jobs(seed: int = 4):
    from paper_1303_5164_gb300.tenants import MIX_TYPES
    return [(nm, seed, 8 * b + i, serve_size(nm, sc)) for b, sc in enumerate(SERVE_SCALES)
            for i, nm in enumerate(MIX_TYPES)]


def generate(jobs, workers: int):
    # spawn: the pool starts before any CUDA call and shares nothing with it
    if workers <= 1:
        return [_gen_one(j) for j in jobs]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        return pool.map(_gen_one, jobs, chunksize=1)


# ---------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


class NvmlSampler:
    """SM clock and clock-event reasons every 5 ms through NVML (ctypes), for
    timed regions shorter than nvidia-smi's sampling period."""

    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device: int):
        import ctypes
        import threading
        self.ok = False
        self.samples = []
        self._stop = threading.Event()
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if self.nvml.nvmlDeviceGetHandleByIndex_v2(device, ctypes.byref(self.h)) != 0:
                return
            mx = ctypes.c_uint()
            self.max_mhz = mx.value if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 else None
            self.ok = True
        except Exception:
            self.ok = False
        self._thr = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        import ctypes
        mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(mhz)) == 0:
                r = rs.value if self.nvml.nvmlDeviceGetCurrentClocksEventReasons(self.h, ctypes.byref(rs)) == 0 else 0
                self.samples.append((mhz.value, r))
            time.sleep(0.005)

    def __enter__(self):
        if self.ok:
            self._thr.start()
        return self

    def __exit__(self, *a):
        if self.ok:
            self._stop.set()
            self._thr.join(timeout=2)

    def summary(self):
        if not self.ok or not self.samples:
            return None
        mask = 0
        for _, r in self.samples:
            mask |= r
        return {"sm_mhz": statistics.median(m for m, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(v for b, v in self.BITS.items() if mask & b), "samples": len(self.samples)}


# ---------------------------------------------------------------------- helpers

def _pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


PROFILES = os.path.join(ROOT, "paper_1303_5164_gb300", "profiles_gb300.json")
# DRAM bytes of one co-scheduler launch on a small case (one instance of each
# mix type), with the factor that scales it to the bench's launch
TRAFFIC = os.path.join(ROOT, "profiles", "cosched_kernel_mix_dram.txt")
KERNEL_SOURCES = ["kl_cosched.cu", "tenants.cuh", "kl_internal.h"]


def kernel_source_hash() -> str:
    """sha256 over the co-scheduler kernel's sources (the counters below are
    only valid for the kernel they were taken on)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1303_5164_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _measured_traffic(workload: str):
    """DRAM bytes per cosched_kernel launch of the bench's workload, from the
    committed ncu summary of a smaller launch scaled by the units it processed,
    or None when it is missing, for another workload, or taken on other sources."""
    if not os.path.exists(TRAFFIC):
        return None
    kv = {}
    with open(TRAFFIC) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("workload") != workload or kv.get("kernel_source_sha256") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _load_profiles(K, path=PROFILES):
    """Measured per-type model inputs and slice sizes, if a profile file exists."""
    if not path or not os.path.exists(path):
        return None, None
    with open(path) as f:
        d = json.load(f)
    profs = []
    for t, name in enumerate(K.TYPE_NAMES):
        p = K.kl_profile()
        e = d.get("types", {}).get(name)
        if e:
            for k in ("R_m", "f_u", "m_c", "m_u", "L0", "I_block", "PUR", "MUR"):
                setattr(p, k, float(e[k]))
            p.warps_per_block = int(e.get("warps_per_block", 8))
            p.slice_blocks = int(d.get("slices", {}).get(name, 0))
            p.slice_blocks_alone = int(d.get("slice_autotune_alone", {}).get("slices", {}).get(name, 0))
            p.valid = 1
        profs.append(p)
    return profs, d


def _oracle_one(name, inp):
    """One tenant instance through the CPU oracle (its C loops run with the
    GIL released, so threads calling this run on separate cores)."""
    from oracle import tenants as OT
    if name == "gemm_f32":
        OT.gemm_f32(inp["A"], inp["B"])
    elif name == "spmv_csr":
        OT.spmv_csr(inp["rowptr"], inp["col"], inp["val"], inp["x"])
    elif name == "blackscholes":
        OT.blackscholes(inp["S"], inp["K"], inp["r"], inp["v"], inp["T"])
    elif name == "pchase":
        OT.pchase(inp["next"], inp["start"], inp["hops"])
    elif name == "triad":
        OT.triad(inp["b"], inp["c"], inp["s"])
    elif name == "hist256":
        OT.hist256(inp["data"])
    elif name == "escape":
        OT.escape(inp["width"], inp["height"], inp["max_iter"], inp["x0"], inp["y0"], inp["dx"], inp["dy"])
    elif name == "bitonic":
        OT.sort_u32(inp["data"])
    elif name == "gather":
        OT.gather(inp["a"], inp["idx"])
    else:
        raise ValueError(name)


def cpu_oracle_sample(jobs_inputs):
    """The CPU oracle on one instance of each tenant type (single thread)."""
    from oracle import tenants as OT
    OT.build()
    seen = {}
    for (name, inp) in jobs_inputs:
        if name not in seen:
            seen[name] = inp
    t0 = time.perf_counter()
    for name, inp in seen.items():
        _oracle_one(name, inp)
    dt = time.perf_counter() - t0
    return len(seen), dt, sorted(seen)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_all_cores(jobs_inputs, threads: int | None = None):
    """The CPU oracle on every instance of the batch, one instance per task on
    a pool of `threads` host threads (all cores by default): wall time of
    the whole batch. Returns (instances, seconds, threads)."""
    import concurrent.futures as cf
    from oracle import tenants as OT
    OT.build()
    OT.lib()  # load once, before the threads
    threads = threads or host_cores()
    # longest first, so the pool does not end on one long instance
    order = sorted(range(len(jobs_inputs)), key=lambda i: jobs_inputs[i][0] != "gemm_f32")
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda i: _oracle_one(*jobs_inputs[i]), order))
    return len(jobs_inputs), time.perf_counter() - t0, threads


def gpu_numa_node(device: int):
    """NUMA node of the GPU's PCI function (sysfs), or None when unknown."""
    try:
        import torch
        p = torch.cuda.get_device_properties(device)
        dom, bus, dev = (getattr(p, "pci_domain_id", None), getattr(p, "pci_bus_id", None),
                         getattr(p, "pci_device_id", None))
        if bus is None:
            return None
        with open(f"/sys/bus/pci/devices/{dom or 0:04x}:{bus:02x}:{dev or 0:02x}.0/numa_node") as f:
            n = int(f.read().strip())
        return n if n >= 0 else None
    except (OSError, ValueError, RuntimeError):
        return None


def bind_host_to_gpu_node(device: int):
    """Run this process on the host cores of the GPU's NUMA node, so pinned
    buffers allocated afterwards (first touched by this thread) sit in that
    node's memory. Returns (node, cores) or (None, None) when there is no such
    information."""
    node = gpu_numa_node(device)
    if node is None:
        return None, None
    try:
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                lo, hi = part.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif part:
                cpus.add(int(part))
        if not cpus:
            return node, None
        os.sched_setaffinity(0, cpus)
        return node, len(cpus)
    except (OSError, ValueError, AttributeError):
        return node, None


def make_runtime(K, device: int = 0, stream: int = 0, flags=None, profiles: str = "measured"):
    """The runtime the timed co-scheduled steps use: default configuration
    (4096 pending kernels, the library's default flags unless `flags`), the
    measured HBM bandwidth in the model, and the measured per-type profiles
    and fitted latency parameters. Returns (runtime, model params, model info)."""
    cfg = K.config_default()
    cfg.device = device
    cfg.max_tenants = 4096
    if flags is not None:
        cfg.flags = flags
    rt = K.Runtime(cfg, stream=stream)
    hbm_gbs, _ = _measured_peaks()
    mp_ = rt.model_params()
    mp_.dram_bytes_per_s = hbm_gbs * 1e9
    rt.set_model_params(mp_)
    profs, prof_doc = _load_profiles(K, None if profiles == "none" else PROFILES)
    model_info = {"profiles": "built-in (not measured)"}
    if profs:
        rt.set_profiles(profs)
        mp_.a0, mp_.b0 = prof_doc.get("a0", 1.0), prof_doc.get("b0", 0.0)
        rt.set_model_params(mp_)
        model_info = {"profiles": prof_doc.get("source"), "a0": mp_.a0, "b0": mp_.b0,
                      "solo_ipc_mae_per_sm": prof_doc.get("ipc_mae_per_sm"), "ipc_peak_per_sm": 4.0,
                      "slices": prof_doc.get("slices")}
    return rt, mp_, model_info


def e2e_leg(K, T, rt, tens, names, inputs, stream, local, world, steps, barrier):
    """The metric end to end through the public API from pinned host memory.
    Every step uploads its 64 kernels' inputs, runs them (kl_submit_batch,
    kl_launch, kl_drain) and downloads every output. Two device buffer sets
    (step k uses set k % 2) let the upload of step k+1 and the download of
    step k-1 run on their own streams while step k computes; all of every
    step's copies are inside the timed region. Returns the e2e dict, with the
    per-step upload, compute and download times (CUDA events, medians)."""
    import torch
    n = len(tens)
    sets = [tens, [T.make(nm, x) for nm, x in zip(names, inputs)]]
    set_descs = [K.make_descs((t.type, t.args) for t in ts) for ts in sets]
    affinity = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
    numa_node, numa_cores = bind_host_to_gpu_node(local)
    pin_in, pin_out = [], []
    h2d = d2h = 0
    for t in tens:
        ins = {k: v.cpu().pin_memory() for k, v in t.bufs.items() if k not in t.outputs}
        outs = {k: torch.empty(t.bufs[k].shape, dtype=t.bufs[k].dtype, pin_memory=True) for k in t.outputs}
        h2d += sum(v.numel() * v.element_size() for v in ins.values())
        d2h += sum(v.numel() * v.element_size() for v in outs.values())
        pin_in.append(ins)
        pin_out.append(outs)
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def tev():
        return torch.cuda.Event(enable_timing=True)

    ev_in = [torch.cuda.Event(), torch.cuda.Event()]     # inputs of set b uploaded
    ev_done = [torch.cuda.Event(), torch.cuda.Event()]   # compute on set b finished
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]    # outputs of set b downloaded
    spans = {"upload": [], "compute": [], "download": []}
    timeline = []

    def upload(b):
        s_in.wait_event(ev_done[b])          # the previous run on set b no longer reads its inputs
        e0, e1 = tev(), tev()
        e0.record(s_in)
        with torch.cuda.stream(s_in):
            for t, ins in zip(sets[b], pin_in):
                for k, v in ins.items():
                    t.bufs[k].copy_(v, non_blocking=True)
        e1.record(s_in)
        ev_in[b].record(s_in)
        spans["upload"].append((e0, e1))

    def download(b):
        s_out.wait_event(ev_done[b])
        e0, e1 = tev(), tev()
        e0.record(s_out)
        with torch.cuda.stream(s_out):
            for t, outs in zip(sets[b], pin_out):
                for k, v in outs.items():
                    v.copy_(t.bufs[k], non_blocking=True)
        e1.record(s_out)
        ev_out[b].record(s_out)
        spans["download"].append((e0, e1))

    def run(nsteps):
        for v in spans.values():
            v.clear()
        barrier()
        e0, e1 = tev(), tev()
        e0.record(stream)
        s_in.wait_event(e0)
        s_out.wait_event(e0)
        upload(0)
        for k in range(nsteps):
            b = k % 2
            if k + 1 < nsteps:
                upload(1 - b)
            stream.wait_event(ev_in[b])
            stream.wait_event(ev_out[b])     # outputs of set b read back before they are overwritten
            c0, c1 = tev(), tev()
            c0.record(stream)
            rt.submit_batch(set_descs[b])
            rt.launch()
            rc = rt.drain()
            if rc != 0:
                raise RuntimeError(f"co-scheduled run failed: {K.lib().kl_strerror(rc).decode()}")
            c1.record(stream)
            spans["compute"].append((c0, c1))
            ev_done[b].record(stream)
            download(b)
        for b in range(min(2, nsteps)):
            stream.wait_event(ev_out[b])
        e1.record(stream)
        barrier()
        # where each step's spans sit on the run's clock (ms from its start)
        timeline.clear()
        for k in range(min(nsteps, 6)):
            timeline.append({n: [round(e0.elapsed_time(v[k][0]), 2), round(e0.elapsed_time(v[k][1]), 2)]
                             for n, v in spans.items() if k < len(v)})
        return max_over_ranks(e0.elapsed_time(e1) / nsteps, world, "cuda")

    run(2)
    ms = run(steps)
    per = {k: statistics.median(a.elapsed_time(b) for a, b in v) for k, v in spans.items() if v}

    def copy_gbs(upload_dir):
        # one step's copies alone, on one stream: the link's achieved rate
        q = torch.cuda.Stream()
        c0, c1 = tev(), tev()
        torch.cuda.synchronize()
        c0.record(q)
        with torch.cuda.stream(q):
            for t, ins, outs in zip(tens, pin_in, pin_out):
                if upload_dir:
                    for k, v in ins.items():
                        t.bufs[k].copy_(v, non_blocking=True)
                else:
                    for k, v in outs.items():
                        v.copy_(t.bufs[k], non_blocking=True)
        c1.record(q)
        c1.synchronize()
        return (h2d if upload_dir else d2h) / (c0.elapsed_time(c1) / 1e3) / 1e9

    h2d_gbs, d2h_gbs = copy_gbs(True), copy_gbs(False)
    if affinity is not None:
        os.sched_setaffinity(0, affinity)
    return {"value": job_value(n, world, ms), "unit": "kernels/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms,
            "step_ms_median": {k: round(v, 3) for k, v in per.items()},
            "timeline_ms": timeline,
            "h2d_gbs_alone": h2d_gbs, "d2h_gbs_alone": d2h_gbs,
            "host_numa_node": numa_node, "host_cores_bound": numa_cores,
            "how": "public API (kl_submit_batch/kl_launch/kl_drain) on pinned host buffers; uploads and downloads on "
                   "their own streams, overlapping the neighbouring steps' compute (two device buffer sets); "
                   "pinned buffers allocated with the process bound to the GPU's NUMA node (when sysfs "
                   "names one); step_ms_median = each stream's span per step; *_gbs_alone = one step's copies "
                   "in one direction, alone on one stream"}


# ---------------------------------------------------------------------- reference arm

def run_reference(args):
    """The CPU oracle as the reference arm: each step runs the whole 64-kernel
    mix (the same kernels, sizes and order the co-scheduled arm times) on all
    host cores, one kernel instance per thread-pool task."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    jobs = mix_jobs()
    inputs = generate(jobs, max(1, min(len(jobs), host_cores())))
    pairs = [(j[0], x) for j, x in zip(jobs, inputs)]
    for _ in range(args.warmup):
        cpu_oracle_all_cores(pairs)
    times = []
    for _ in range(args.steps):
        n, dt, cores = cpu_oracle_all_cores(pairs)
        times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    val = n / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "kernels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+i32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "kernels_per_step": n,
                       "reference": f"CPU oracle (oracle/tenants.c) on {cores} host threads"},
            "cpu_baseline": {"value": val, "unit": "kernels/s", "cores": cores, "kind": "oracle",
                             "sample": f"the whole {n}-kernel mix per step, full size, one instance per "
                                       f"task on {cores} threads"},
            "e2e": {"value": val, "unit": "kernels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------- our arm

def run_ours(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    jobs = mix_jobs() if args.workload == "mix" else batch_jobs()
    t_gen = time.time()
    inputs = generate(jobs, max(1, min(len(jobs), (os.cpu_count() or 2) // max(1, world))))
    t_gen = time.time() - t_gen

    import numpy as np
    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1303_5164_gb300 import build as kb
    from paper_1303_5164_gb300 import kernelet as K
    from paper_1303_5164_gb300 import roofline as RF
    from paper_1303_5164_gb300 import tenants as T
    kb.build()

    names = [j[0] for j in jobs]
    tens = [T.make(nm, x) for nm, x in zip(names, inputs)]
    stream = torch.cuda.current_stream()
    rt, mp_, model_info = make_runtime(K, local, stream.cuda_stream, args.flags, args.profiles)
    hbm_gbs, peak_src = _measured_peaks()
    prof_src = model_info["profiles"]

    descs = K.make_descs((t.type, t.args) for t in tens)

    def launcher(mode, ns=0):
        if mode is None:
            return rt.launch
        return lambda: rt.launch_baseline(mode, ns)

    def check_run(rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} run failed: {K.lib().kl_strerror(rc).decode()}")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def steps_pipelined(mode, ns, steps, collect=None):
        """`steps` runs of the whole batch, the host work of one step overlapped
        with the previous run: the next batch is submitted (kl_submit_batch)
        while the current run is in flight, kl_wait_run waits for that run only,
        and the next run is launched before the finished one's stats are read.
        Every step's submission, launch and wait are inside the caller's region."""
        launch = launcher(mode, ns)
        hs = rt.submit_batch(descs)
        launch()
        for k in range(steps):
            nxt = rt.submit_batch(descs) if k + 1 < steps else None
            check_run(rt.wait_run(), "co-scheduled" if mode is None else "baseline")
            rs = rt.run_stats() if collect else None   # the run just finished (read before the next retires)
            if nxt is not None:
                launch()
            if collect:
                collect(hs, rs)
            hs = nxt

    def timed(mode, ns, steps, collect=None):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        steps_pipelined(mode, ns, steps, collect)
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / steps, world, "cuda")

    for mode, ns in ((None, 0), (K.KL_BASE_MULTISTREAM, args.nstreams), (K.KL_BASE_SERIAL, 1)):
        steps_pipelined(mode, ns, args.warmup)

    lat_co, kern_ns, phases_n = [], [], []

    def col_co(hs, rs):
        kern_ns.append(rs.kernel_ns)
        phases_n.append(rs.n_phases)
        for h in hs:
            s = rt.stats(h)
            lat_co.append((s.t_end_ns - s.t_launch_ns) / 1e6)

    lat_ms = []

    def col_ms(hs, rs):
        for h in hs:
            lat_ms.append(rt.stats(h).t_end_ns / 1e6)

    with ClockSampler(local) as clk, NvmlSampler(local) as nv:
        ms_co = timed(None, 0, args.steps, col_co)
    clocks = clk.summary()
    nvs = nv.summary()
    if nvs:
        clocks = dict(nvs, nvidia_smi=clocks)
    ms_ms = timed(K.KL_BASE_MULTISTREAM, args.nstreams, args.steps, col_ms)
    ms_se = timed(K.KL_BASE_SERIAL, 1, args.steps)

    n = len(tens)
    value = job_value(n, world, ms_co)

    # roofline of the dominant (only) kernel: the persistent co-scheduler
    esc_iters = {}
    for t in tens:
        if t.name == "escape":
            esc_iters[id(t)] = int(t.bufs["count"].to(torch.int64).sum().item())
    bytes_mix = sum(RF.algo_bytes(nm, x) for nm, x in zip(names, inputs))
    flops_mix = sum(RF.fp32_flops(nm, x, esc_iters.get(id(t))) for nm, x, t in zip(names, inputs, tens))
    ops_mix = sum(RF.lane_ops(nm, x, esc_iters.get(id(t))) for nm, x, t in zip(names, inputs, tens))
    kern_ms = statistics.median(kern_ns) / 1e6
    achieved = bytes_mix / (kern_ms / 1e3) / 1e9
    f_sm = (clocks.get("sm_mhz") or 1900.0) * 1e6
    t_hbm = bytes_mix / (hbm_gbs * 1e9)
    t_issue = ops_mix / RF.lane_peak(mp_.n_sm, f_sm)
    t_roof = max(t_hbm, t_issue)

    # end to end through the public API with host buffers: H2D inputs, run, D2H outputs
    e2e = None
    if not args.no_e2e:
        e2e = e2e_leg(K, T, rt, tens, names, inputs, stream, local, world, max(4, args.steps), barrier)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        pairs = list(zip(names, inputs))
        k, dt, cores = cpu_oracle_all_cores(pairs)
        k1, dt1, kinds = cpu_oracle_sample(pairs)
        cpu = {"value": k / dt, "unit": "kernels/s", "cores": cores, "kind": "oracle",
               "sample": f"the whole {k}-kernel mix, full size, one instance per task on {cores} host "
                         f"threads, {dt:.1f} s",
               "single_thread": {"value": k1 / dt1, "unit": "kernels/s", "cores": 1,
                                 "sample": f"one full-size instance of each of the {k1} kernel types "
                                           f"({', '.join(kinds)}), {dt1:.1f} s"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "kernels/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_co, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+i32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.workload == "mix" else BATCH_WORKLOAD, "kernels_per_step": n, "l2": "inputs larger than L2 (about "
                       f"{bytes_mix / 1e9:.1f} GB touched per step)", "slots_per_sm": rt.run_stats().slots_per_sm,
                       "multistream_streams": args.nstreams, "profiles": prof_src,
                       "host_overlap": "every arm submits the next batch (one kl_submit_batch call) while "
                                       "the current run is in flight and waits with kl_wait_run",
                       "parallelism": f"replicas x{world}"},
            "speedup_vs_multistream": ms_ms / ms_co, "speedup_vs_serial": ms_se / ms_co,
            "multistream_kernels_per_s": world * n / (ms_ms / 1e3), "serial_kernels_per_s": world * n / (ms_se / 1e3),
            "makespan_ms": {"cosched": ms_co, "multistream": ms_ms, "serial": ms_se},
            "latency_ms": {"cosched_p50": _pct(lat_co, 50), "cosched_p99": _pct(lat_co, 99),
                           "multistream_p50": _pct(lat_ms, 50), "multistream_p99": _pct(lat_ms, 99)},
            "mix_roofline": {"t_roof_ms": t_roof * 1e3, "frac": (t_roof * 1e3) / kern_ms,
                             "t_hbm_ms": t_hbm * 1e3, "t_issue_ms": t_issue * 1e3,
                             "algo_bytes": bytes_mix, "lane_ops": ops_mix, "fp32_flops": flops_mix,
                             "how": "T_roof = max(sum of algorithmic bytes / measured HBM, sum of lane "
                                    "operations / (SMs x 128 lanes x sampled SM clock))"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
                         "frac": achieved / hbm_gbs, "traffic": _measured_traffic(args.workload),
                         "kernel": "cosched_kernel", "kernel_ms": kern_ms,
                         "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                         else "fallback 6800 GB/s"},
            "phases_per_run": statistics.median(phases_n) if phases_n else None,
            "model": model_info,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            # per timed step: the run image staged in, the co-scheduler, the results staged out
            "gpu_launches": 3 * args.steps,
            "input_gen_s": round(t_gen, 1),
        }
        print(json.dumps(line))
    rt.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """Open-loop serving sweep: for each offered rate, Poisson arrivals for
    --serve-seconds; an arrival waits in the client's FIFO until the runtime
    admits it (kl_submit returns KL_EAGAIN while the in-flight slots or the
    footprint cap are full) and a free output replica of its (type, size)
    exists. Latency = arrival to the host seeing the completion. The same
    arrival sequence drives the co-scheduled server and the plain multi-stream
    FIFO server."""
    import numpy as np
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    jobs = serve_jobs()
    t_gen = time.time()
    inputs = generate(jobs, max(1, min(len(jobs), (os.cpu_count() or 2) // max(1, world))))
    t_gen = time.time() - t_gen
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1303_5164_gb300 import build as kb
    from paper_1303_5164_gb300 import kernelet as K
    from paper_1303_5164_gb300 import tenants as T
    kb.build()
    from paper_1303_5164_gb300.tenants import MIX_TYPES
    base = [T.make(j[0], x) for j, x in zip(jobs, inputs)]
    del inputs
    reps = [[t] + [t.replica() for _ in range(args.serve_replicas - 1)] for t in base]
    descs = [[K.make_desc(t.type, t.args, 0, t.footprint) for t in r] for r in reps]
    torch.cuda.synchronize()
    dev_gb = torch.cuda.memory_allocated() / 1e9
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    cfg = K.config_default()
    cfg.device = local
    cfg.max_tenants = 4 * n_sm
    if args.flags is not None:
        cfg.flags = args.flags
    cfg.mem_cap_bytes = 150 * 10**9
    stream = torch.cuda.Stream()  # the serving kernel holds its stream for the whole run
    rt = K.Runtime(cfg, stream=stream.cuda_stream)
    hbm_gbs, _ = _measured_peaks()
    mp_ = rt.model_params()
    mp_.dram_bytes_per_s = hbm_gbs * 1e9
    rt.set_model_params(mp_)
    profs, prof_doc = _load_profiles(K, None if args.profiles == "none" else PROFILES)
    if profs:
        rt.set_profiles(profs)
        mp_.a0, mp_.b0 = prof_doc.get("a0", 1.0), prof_doc.get("b0", 0.0)
        rt.set_model_params(mp_)
    lib = K.lib()
    import ctypes as C
    hbuf = (K.U64 * 8192)()
    nbuf = K.U32()

    def one_rate(rate, mode, seed):
        rng = np.random.default_rng(seed)
        n_arr = max(1, int(rng.poisson(rate * args.serve_seconds)))
        t_arr = np.sort(rng.uniform(0.0, args.serve_seconds, n_arr))
        kinds = rng.integers(0, len(MIX_TYPES), n_arr)
        buckets = rng.choice(len(SERVE_SCALES), n_arr, p=SERVE_P)
        combo = buckets * len(MIX_TYPES) + kinds
        free = [list(range(args.serve_replicas)) for _ in base]
        owner = {}
        lat, done_t = [], []
        if mode == "cosched":
            rt.serve_start(K.KL_SERVE_COSCHED, 0, 0)
        else:
            rt.serve_start(K.KL_BASE_MULTISTREAM, args.nstreams, 0)
        h = C.c_uint64()
        nxt = 0
        t0 = time.perf_counter()
        t_end = t0 + args.serve_seconds
        while True:
            now = time.perf_counter()
            rc = lib.kl_reap(rt._h, hbuf, 8192, C.byref(nbuf))
            if rc:
                raise RuntimeError(f"kl_reap: {rc}")
            for i in range(nbuf.value):
                k, c, r = owner.pop(hbuf[i])
                free[c].append(r)
                lat.append(now - t0 - t_arr[k])
                done_t.append(now - t0)
            if now >= t_end:
                break
            while nxt < n_arr and t_arr[nxt] <= now - t0:
                c = int(combo[nxt])
                if not free[c]:
                    break          # FIFO: the head waits for an output replica
                r = free[c][-1]
                rc = lib.kl_submit(rt._h, C.byref(descs[c][r]), C.byref(h))
                if rc == K.KL_EAGAIN:
                    break          # FIFO: the head waits for admission
                if rc:
                    raise RuntimeError(f"kl_submit: {lib.kl_strerror(rc).decode()}")
                free[c].pop()
                owner[h.value] = (nxt, c, r)
                nxt += 1
        admitted, in_flight = nxt, len(owner)
        # arrivals are over: finish what was admitted (not counted as in-window throughput)
        rc = rt.serve_stop(60_000_000_000)
        if rc:
            raise RuntimeError(f"serve run failed: {lib.kl_strerror(rc).decode()}")
        done_in = len(done_t)
        return {"offered_per_s": rate, "arrivals": n_arr, "admitted": admitted, "completed_in_window": done_in,
                "throughput_per_s": done_in / args.serve_seconds,
                "p50_ms": 1e3 * _pct(lat, 50) if lat else None, "p99_ms": 1e3 * _pct(lat, 99) if lat else None,
                "not_admitted": n_arr - admitted, "in_flight_at_end": in_flight}

    rates = [float(x) for x in args.serve_rates.split(",")]
    # warm-up: a short run of each server
    keep = args.serve_seconds
    args.serve_seconds = 0.3
    for _ in range(max(1, args.warmup // 3)):
        one_rate(1000.0, "cosched", 1)
        one_rate(1000.0, "multistream", 1)
    args.serve_seconds = keep
    res = {"cosched": [], "multistream": []}
    with ClockSampler(local) as clk, NvmlSampler(local) as nv:
        for i, rate in enumerate(rates):
            for mode in ("cosched", "multistream"):
                res[mode].append(one_rate(rate, mode, 100 + i))
                if rank == 0:
                    print(mode, json.dumps(res[mode][-1]), file=sys.stderr, flush=True)
    clocks = clk.summary()
    nvs = nv.summary()
    if nvs:
        clocks = dict(nvs, nvidia_smi=clocks)
    best = max(res["cosched"], key=lambda r: r["throughput_per_s"])
    best_ms = max(res["multistream"], key=lambda r: r["throughput_per_s"])
    if rank == 0:
        line = {
            "metric": METRIC, "value": world * best["throughput_per_s"], "unit": "kernels/s",
            "n_gpus": world, "steps": len(rates), "warmup": args.warmup,
            "ms_per_step": 1e3 * args.serve_seconds, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+i32", "data": "synthetic",
            "config": {"workload": SERVE_WORKLOAD, "seconds_per_rate": args.serve_seconds,
                       "rates_per_s": rates, "output_replicas": args.serve_replicas,
                       "in_flight_slots": cfg.max_tenants, "mem_cap_bytes": cfg.mem_cap_bytes,
                       "device_gb_allocated": round(dev_gb, 1), "multistream_streams": args.nstreams,
                       "l2": "inputs larger than L2", "parallelism": f"replicas x{world}"},
            "speedup_vs_multistream": best["throughput_per_s"] / best_ms["throughput_per_s"],
            "serve": res, "clocks": clocks, "gpu_launches": 2 * len(rates),
            "input_gen_s": round(t_gen, 1),
        }
        print(json.dumps(line))
    rt.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nstreams", type=int, default=32)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profiles", default="measured", choices=["measured", "none"])
    ap.add_argument("--workload", default="mix", choices=["mix", "batch", "serve"],
                    help="mix: 64 kernels of the eight types; batch: 512 tenants, log-uniform grids; "
                         "serve: open-loop arrival-rate sweep")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-rates", default="100,300,1000,3000,10000,20000")
    ap.add_argument("--serve-replicas", type=int, default=24)
    ap.add_argument("--flags", type=int, default=None, help="kl_config.flags (default: the library's)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
