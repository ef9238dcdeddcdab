#!/usr/bin/env python
"""Benchmark of the GB300 label-propagation path (one JSON line on rank 0).

A step is one whole run of the hot path on one synthetic graph resident in HBM:
lpa_run (label init, sweeps until the tolerance test or the 20-sweep cap, Pick-Less every
4th sweep) followed by lpa_modularity (float64 Eq. 1).  The default workload is the R-MAT
scale-26 graph (67,108,864 vertices, edge factor 16, a,b,c,d = .57,.19,.19,.05,
symmetrised, ~2.1 B CSR entries, int64 offsets, int32 indices, unit float32 weights).

  value   CSR entries scanned per second over the step (sum over sweeps / device time)
  e2e     the same metric through the public API with host buffers: lpa_create from pinned
          host arrays (H2D inside), lpa_run, lpa_labels to host, lpa_modularity, destroy
  roofline  dominant kernel: algorithmic bytes / its CUDA-event time, against measured HBM
  cpu_baseline  the CPU oracle (single thread) on a stratified sample of the first sweep

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload rmat26|rmat22|sbm]
Under torchrun (N > 1) every rank runs an independent replica (the path has no exchange
step across graphs): value = all ranks' entries / max-over-ranks time, scaling "weak".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import torch  # noqa: E402

WORKLOADS = {
    "rmat26": dict(kind="rmat", scale=26, weights="unit",
                   desc="R-MAT scale 26, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), symmetrised, no self-loops/"
                        "duplicates, unit float32 weights, int64 offsets"),
    "rmat22": dict(kind="rmat", scale=22, weights="int8",
                   desc="R-MAT scale 22, edge factor 16, (a,b,c,d)=(.57,.19,.19,.05), symmetrised, integer "
                        "weights 1..8 as float32"),
    "rmat22u": dict(kind="rmat", scale=22, weights="unit",
                    desc="R-MAT scale 22 with unit float32 weights: the smaller case on which the counters behind "
                         "the R-MAT 26 roofline's traffic are captured"),
    "sbm": dict(kind="sbm", n=10_000, block=100, d_in=16.0, d_out=2.0, weights="unit",
                desc="planted partition 10,000 vertices / 100 blocks, intra-degree 16, inter-degree 2, unit weights"),
}
ALG = dict(tolerance=0.05, max_iters=20, pl_period=4)
BYTES_PER_EDGE_W = 12      # neighbour index 4 + weight 4 + gathered label 4
BYTES_PER_EDGE_U = 8       # unit weights (NULL, or all exactly 1: not read): index 4 + label 4
BYTES_PER_VERTEX = 17      # offsets 2x4 (amortised) + own label 4 + label write 4 + flag 1


# DRAM bytes per scanned CSR entry of each kernel slot (all launches of the slot over one run,
# read + write, divided by the entries the slot scanned in that run), from one ncu capture of
# the counters on R-MAT 22 with unit weights, a case small enough to capture with counters.  The
# traffic reported for a launch of a larger graph is that rate times the entries the launch
# scans: a scaled figure, not a measurement of the larger graph (its label gathers miss L2 more
# often than R-MAT 22's).  Reported while the sweep sources hash as they did at capture time.
TRAFFIC = {
    "captured_on": "rmat22u",
    "bytes_per_entry": {"cta": 4.66, "cta_large": 4.7, "group": 11.56, "hub_acc": 8.53, "thread": 29.78, "warp": 6.41},
    "sources": {
        "sweep_kernels.cuh": "01c8c54c550a37545072c04afdea60ee675cdc1a5d0ea5dace66c75d9e61f914",
        "lpa_sweep.cu": "b1f909ed0f74c9a5cff959a0ef8aa187f877483c72afdf1deff10792cacfdd89",
        "lpa_internal.h": "0442f8cc30d379d5cf49344867d65e0da6bdb86ff3167529751b844c7755ea60",
        "lpa_graph.cu": "8380a25d7f40eff4bcfba751b70b736f19fb830ebcc51b35e108d2c0047416b1",
    },
}


def traffic_for(kernel: str, entries_per_launch: float):
    """Scaled DRAM bytes per launch of a kernel slot, or None (no rate, or sources changed)."""
    import hashlib
    rate = TRAFFIC["bytes_per_entry"].get(kernel)
    if rate is None or not TRAFFIC["sources"]:
        return None
    csrc = os.path.join(ROOT, "paper_2411_11468_gb300", "csrc")
    for name, digest in TRAFFIC["sources"].items():
        try:
            with open(os.path.join(csrc, name), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return rate * entries_per_launch


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def over_ranks(x: float, op: str, device=None) -> float:
    """x reduced over the ranks of the default process group ("max" or "sum"); x itself
    without a group.  The replicas' step time is the maximum over ranks, their work the sum."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def make_graph(name, device):
    from paper_2411_11468_gb300 import graphgen as gg
    w = WORKLOADS[name]
    if w["kind"] == "rmat":
        return gg.rmat(w["scale"], weights=w["weights"], device=device)
    return gg.sbm(w["n"], w["block"], w["d_in"], w["d_out"], seed=0, weights=w["weights"], device=device)


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = None
        self.dev = device_index

    def start(self):
        try:
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else ("GPU-" + uuid)]
        except Exception:
            sel = ["-i", str(self.dev)]
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", *sel, f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "power_w_max": max(r["power"] for r in rows)}


def kernel_bytes(stats_dict, weighted: bool):
    """Algorithmic bytes per kernel slot summed over the run (sweep kernels only)."""
    from paper_2411_11468_gb300 import lpa
    per_edge = BYTES_PER_EDGE_W if weighted else BYTES_PER_EDGE_U
    tot = [0.0] * lpa.NUM_KERNELS
    for it in range(len(stats_dict.get("kernel_edges", []))):
        for k in range(lpa.NUM_KERNELS):
            tot[k] += per_edge * stats_dict["kernel_edges"][it][k] + BYTES_PER_VERTEX * stats_dict["kernel_active"][it][k]
    return tot


def cpu_baseline(csr_dev, n_windows=16, target_s=12.0):
    """The oracle's synchronous first sweep (all vertices active, Pick-Less on) over a
    stratified sample of vertex windows; returns edges/s, time and the sample description."""
    import numpy as np

    import oracle
    off = csr_dev.offsets
    n = off.numel() - 1
    labels = np.arange(n, dtype=np.int32)

    def window(v0, target_edges):
        o0 = int(off[v0])
        hi = int(torch.searchsorted(off, torch.tensor([o0 + target_edges], device=off.device)).item())
        v1 = max(v0 + 1, min(n, hi))
        return v0, v1

    def run(windows):
        t = 0.0
        edges = 0
        for v0, v1 in windows:
            o0, o1 = int(off[v0]), int(off[v1])
            ow = off[v0:v1 + 1].cpu().numpy()
            iw = csr_dev.indices[o0:o1].cpu().numpy()
            ww = None if csr_dev.weights is None else csr_dev.weights[o0:o1].cpu().numpy()
            t0 = time.perf_counter()
            _, e = oracle.sweep_window(v0, v1, ow, iw, ww, labels, pl=True)
            t += time.perf_counter() - t0
            edges += e
        return edges, t

    starts = [int(k * n // n_windows) for k in range(n_windows)]
    probe = [window(v, 20_000) for v in starts]
    e, t = run(probe)
    rate = e / max(t, 1e-9)
    per_window = int(max(50_000, rate * target_s / n_windows))
    wins = [window(v, per_window) for v in starts]
    e, t = run(wins)
    nverts = sum(v1 - v0 for v0, v1 in wins)
    return dict(value=e / t, unit="edges/s", cores=1, kind="oracle", seconds=round(t, 3),
                sample=f"first synchronous sweep (Pick-Less, all vertices active) over {n_windows} vertex windows "
                       f"evenly spaced in id order: {nverts} vertices, {e} CSR entries; single-threaded C oracle",
                host=dict(machine=platform.machine(), nproc=os.cpu_count(), cpu=_cpu_model()))


def swap_sbm(lpa, dev):
    """Section 4.1's comparison on the planted partition (10,000 vertices, 100 blocks):
    iterations, modularity and run time for Pick-Less / Cross-Check periods, synchronous."""
    from paper_2411_11468_gb300 import graphgen as gg
    w = WORKLOADS["sbm"]
    csr = gg.sbm(w["n"], w["block"], w["d_in"], w["d_out"], seed=0, weights=w["weights"], device=dev)
    g = lpa.Graph(csr.offsets, csr.indices, csr.weights)
    out = {}
    for name, pl, cc in (("none", 0, 0), ("PL1", 1, 0), ("PL4", 4, 0), ("CC1", 0, 1), ("CC2", 0, 2),
                         ("CC4", 0, 4), ("PL4+CC4", 4, 4), ("PL2+CC2", 2, 2)):
        best = None
        for _ in range(3):
            st = g.run(ALG["tolerance"], ALG["max_iters"], pl, lpa.SYNC, cc_period=cc).to_dict()
            best = st if best is None or st["total_ms"] < best["total_ms"] else best
        out[name] = {"run_ms": round(best["total_ms"], 3), "iterations": best["iterations"],
                     "converged": best["converged"], "modularity": round(g.modularity(), 5)}
    g.close()
    return out


def cpu_multicore(csr_dev, h_off=None, h_idx=None, h_w=None, full=False):
    """The multicore CPU baseline (OpenMP restatement of the synchronous run, all host cores):
    the first, all-active sweep of the whole graph in entries/s, and with full=True the whole
    run too (returned with its result, for the parity check)."""
    import oracle
    if h_off is None:
        h_off, h_idx = csr_dev.offsets.cpu(), csr_dev.indices.cpu()
        h_w = None if csr_dev.weights is None else csr_dev.weights.cpu()
    og = oracle.Graph(h_off, h_idx, h_w)
    threads = oracle.multicore_threads()
    t0 = time.perf_counter()
    r = oracle.multicore_lpa_sync(og, ALG["tolerance"], 1, ALG["pl_period"])
    t = time.perf_counter() - t0
    out = dict(value=r.edges[0] / t, unit="edges/s", cores=threads, kind="multicore", seconds=round(t, 3),
               moved=r.dN[0] if r.dN else 0,
               sample=f"first synchronous sweep (Pick-Less, all vertices active) over the whole graph: {og.n} "
                      f"vertices, {og.m} CSR entries; OpenMP over {threads} threads, per-thread hash tables")
    if not full:
        return out
    t0 = time.perf_counter()
    rf = oracle.multicore_lpa_sync(og, ALG["tolerance"], ALG["max_iters"], ALG["pl_period"])
    tf = time.perf_counter() - t0
    out["full_run"] = dict(seconds=round(tf, 3), sweeps=rf.iterations, edges=sum(rf.edges),
                           value=sum(rf.edges) / tf, unit="edges/s")
    return out, rf


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor()


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    if args.workload in ("batch", "serve"):
        return run_reference_multi(args)
    device = "cuda" if torch.cuda.is_available() else "cpu"
    csr = make_graph(args.workload, device)
    w = WORKLOADS[args.workload]
    vals = []
    for step in range(args.warmup + args.steps):
        r = cpu_baseline(csr, target_s=args.ref_seconds)
        if step >= args.warmup:
            vals.append(r)
    value = statistics.median(v["value"] for v in vals)
    ms = statistics.median(v["seconds"] for v in vals) * 1000.0
    line = {"impl": "reference", "metric": metric_name(args.workload), "value": value, "unit": "edges/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "graph": w["desc"], "mode": args.mode, **ALG},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": vals[-1]["sample"], "value": value,
                             "unit": "edges/s", "host": vals[-1]["host"]},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_multi(args):
    """The oracle (synchronous, single thread) on the batched or served workload's graphs, in
    order, until about --ref-seconds of oracle time per step: graphs or requests per second."""
    import oracle
    from paper_2411_11468_gb300 import graphgen as gg
    import numpy as np
    if args.workload == "batch":
        specs = gg.batch_specs(args.batch_graphs)
        make = lambda k: gg.batch_graph(specs[k], weights="unit")
        order = list(range(len(specs)))
        unit, metric = "graphs/s", "batched LPA graphs solved per second (4,096 SBM graphs)"
    else:
        specs = gg.serve_specs(args.serve_pool)
        make = lambda k: gg.serve_graph(specs[k])
        rng = np.random.default_rng(12345)
        order = [int(x) for x in rng.integers(0, len(specs), args.serve_requests)]
        unit, metric = "requests/s", "served LPA requests per second (Poisson stream, continuous batching)"
    vals, secs, counts = [], [], []
    pos = 0
    for step in range(args.warmup + args.steps):
        t, k = 0.0, 0
        while t < args.ref_seconds and k < len(order):
            g = oracle.Graph.of(make(order[(pos + k) % len(order)]))
            t0 = time.perf_counter()
            oracle.lpa_sync(g, ALG["tolerance"], ALG["max_iters"], ALG["pl_period"])
            t += time.perf_counter() - t0
            k += 1
        pos += k
        if step >= args.warmup:
            vals.append(k / t)
            secs.append(t)
            counts.append(k)
    value = statistics.median(vals)
    sample = (f"the first {sum(counts)} {'graphs' if args.workload == 'batch' else 'requests'} of the workload in "
              f"order, whole synchronous runs (tolerance 0.05, cap 20, Pick-Less every 4th sweep), single-threaded C "
              f"oracle, about {args.ref_seconds:.0f} s of oracle time per step; graph generation not timed")
    line = {"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": dist_env()[0],
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(secs) * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "mode": "sync", **ALG},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": value, "unit": unit,
                             "host": dict(machine=platform.machine(), nproc=os.cpu_count(), cpu=_cpu_model())},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def metric_name(workload):
    return f"LPA CSR entries scanned per second, full run to convergence ({workload})"


def roofline_of(stats, weighted, peak, peak_src, workload, steps):
    """Dominant kernel (largest CUDA-event time over the instrumented steps) with its
    algorithmic bytes / time, and the same for the first, all-active sweep."""
    from paper_2411_11468_gb300 import lpa
    kms = [0.0] * lpa.NUM_KERNELS
    kbytes = [0.0] * lpa.NUM_KERNELS
    klaunch = [0] * lpa.NUM_KERNELS
    kentries = [0] * lpa.NUM_KERNELS
    for s in stats:
        kb = kernel_bytes(s, weighted)
        for it in range(len(s["kernel_ms"])):
            for k in range(lpa.NUM_KERNELS):
                if s["kernel_ms"][it][k] > 0:
                    kms[k] += s["kernel_ms"][it][k]
                    klaunch[k] += 1
                    kentries[k] += s["kernel_edges"][it][k]
        for k in range(lpa.NUM_KERNELS):
            kbytes[k] += kb[k]
    dom = max(range(lpa.NUM_KERNELS), key=lambda k: kms[k])
    achieved = kbytes[dom] / (kms[dom] / 1000.0) / 1e9 if kms[dom] > 0 else 0.0
    last = stats[-1]
    per_edge = BYTES_PER_EDGE_W if weighted else BYTES_PER_EDGE_U
    sweep0_ms = last["iter_ms"][0] if last["iter_ms"] else 0.0
    sweep0_bytes = per_edge * last["edges"][0] + BYTES_PER_VERTEX * last["active"][0] if last["edges"] else 0
    kernel_table = {lpa.KERNEL_NAMES[k]: dict(ms_per_step=round(kms[k] / steps, 4), launches_per_step=klaunch[k] / steps,
                                              gbs=round(kbytes[k] / (kms[k] / 1000.0) / 1e9, 1) if kms[k] > 0 else None)
                    for k in range(lpa.NUM_KERNELS) if kms[k] > 0}
    first = None
    if sweep0_ms > 0:
        first = {"ms": round(sweep0_ms, 3), "edges": last["edges"][0],
                 "edges_per_s": last["edges"][0] / (sweep0_ms / 1000.0),
                 "gbs": round(sweep0_bytes / (sweep0_ms / 1000.0) / 1e9, 1),
                 "frac": round(sweep0_bytes / (sweep0_ms / 1000.0) / 1e9 / peak, 4)}
    return {"bound": "hbm", "kernel": lpa.KERNEL_NAMES[dom], "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": traffic_for(lpa.KERNEL_NAMES[dom], kentries[dom] / max(1, klaunch[dom])),
            "traffic_note": f"DRAM bytes per scanned entry captured on {TRAFFIC['captured_on']}, scaled by the "
                            "entries one launch scans", "peak_source": peak_src,
            "bytes_model": f"{per_edge} B per scanned entry + {BYTES_PER_VERTEX} B per processed vertex",
            "first_sweep": first, "kernels": kernel_table}


def oracle_full_run(csr_dev, mode, waves_tuning=None):
    """The single-threaded oracle's whole run (tolerance 0.05, cap 20, Pick-Less every 4th):
    synchronous, or asynchronous in sequential id order; with waves_tuning also the
    asynchronous run under the wave model of the GPU's schedule.  Returns the results and
    the timed seconds of the first run."""
    import oracle
    og = oracle.Graph.of(csr_dev)
    fn = oracle.lpa_sync if mode == "sync" else oracle.lpa_async
    t0 = time.perf_counter()
    r = fn(og, ALG["tolerance"], ALG["max_iters"], ALG["pl_period"])
    secs = time.perf_counter() - t0
    rw = None
    if waves_tuning is not None:
        from oracle.schedule import gpu_schedule
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        waves, takes = gpu_schedule(og.off, waves_tuning, sms)
        rw = oracle.lpa_async_waves(og, waves, ALG["tolerance"], ALG["max_iters"], ALG["pl_period"], take_of=takes)
    return og, r, secs, rw


_CPU_SAMPLE = {}     # the oracle's sampled first-sweep rate, taken once per workload


def measure_single(args, lpa, dev, workload, mode_name, steps, warmup, e2e_steps, extras=False):
    """One workload and mode: the timed steps (uninstrumented), an instrumented pass of the same
    steps for the per-kernel breakdown, parity against the oracle (or the pinned multicore
    baseline), the CPU baseline, end to end from pinned host buffers.  Returns the JSON object."""
    import oracle
    mode = lpa.SYNC if mode_name == "sync" else lpa.ASYNC
    ws, rank, local = dist_env()
    t0 = time.time()
    csr = make_graph(workload, dev)
    torch.cuda.synchronize()
    log(f"[bench] {workload}/{mode_name}: n={csr.n} m={csr.m} generated in {time.time() - t0:.1f}s")
    weighted = csr.weights is not None and not bool(torch.all(csr.weights == 1))   # all-one weights are not read
    stream = torch.cuda.current_stream(dev)
    g = lpa.Graph(csr.offsets, csr.indices, csr.weights)

    def step(time_kernels=False):
        st = g.run(ALG["tolerance"], ALG["max_iters"], ALG["pl_period"], mode, time_kernels=time_kernels)
        q = g.modularity()
        return st, q

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    plain, qs = [], []
    for _ in range(steps):
        st, q = step()
        plain.append(st.to_dict())
        qs.append(q)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = over_ranks(e0.elapsed_time(e1) / steps, "max", dev)
    edges_per_step = over_ranks(statistics.median(sum(s["edges"]) for s in plain), "sum", dev)
    value = edges_per_step / (ms / 1000.0)
    # the same steps with every kernel timed by CUDA events: the per-kernel breakdown
    inst = []
    e0.record(stream)
    for _ in range(steps):
        st_i, q_i = step(time_kernels=True)
        inst.append(st_i.to_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    inst_ms = e0.elapsed_time(e1) / steps
    peak, peak_src = measured_peaks()
    last = plain[-1]
    labels_gpu = g.labels().cpu()
    out = {"metric": metric_name(workload), "value": value, "unit": "edges/s", "n_gpus": ws, "steps": steps,
           "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload, "graph": WORKLOADS[workload]["desc"], "n": csr.n, "m": csr.m,
                      "mode": mode_name, **ALG,
                      "l2": "inputs larger than L2 (CSR resident in HBM)" if csr.m * 4 > 256e6 else
                            "graph smaller than L2: repeated runs read it from L2 (no flush)"},
           "iterations": last["iterations"], "dN": last["changed"], "edges_per_sweep": last["edges"],
           "modularity": q, "processing_rate": ws * csr.m / (ms / 1000.0),
           "roofline": roofline_of(inst, weighted, peak, peak_src, workload, steps),
           "instrumented_ms_per_step": inst_ms,
           "gpu_launches": int(statistics.median(s["launches"] for s in plain)) + 2,
           "clocks": clk, "probe_fallbacks": last["probe_fallbacks"],
           "sweeps": [{"ms": round(inst[-1]["iter_ms"][i], 3), "edges": inst[-1]["edges"][i],
                       "active": inst[-1]["active"][i], "changed": inst[-1]["changed"][i],
                       "kernels": {lpa.KERNEL_NAMES[k]: [round(inst[-1]["kernel_ms"][i][k], 3),
                                                         inst[-1]["kernel_active"][i][k], inst[-1]["kernel_edges"][i][k]]
                                   for k in range(lpa.NUM_KERNELS) if inst[-1]["kernel_ms"][i][k] > 0}}
                      for i in range(len(inst[-1]["iter_ms"]))]}

    if extras and not args.no_ablation and ws == 1:
        out.update(ablations(args, lpa, dev, g, mode))
        g.set_tuning(probe=0, float_values=0)

    # end to end through the public API with host buffers
    h_off = csr.offsets.cpu().pin_memory()
    h_idx = csr.indices.cpu().pin_memory()
    h_w = None if csr.weights is None else csr.weights.cpu().pin_memory()
    if not args.no_e2e:
        h_lab = torch.empty(csr.n, dtype=torch.int32).pin_memory()
        torch.cuda.synchronize()
        times, edges = [], []
        for rep in range(e2e_steps + 1):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            g2 = lpa.Graph(h_off, h_idx, h_w)
            st2 = g2.run(ALG["tolerance"], ALG["max_iters"], ALG["pl_period"], mode)
            g2.labels(h_lab)
            g2.modularity()
            g2.close()
            torch.cuda.synchronize()
            if rep > 0:
                times.append(time.perf_counter() - t1)
                edges.append(sum(st2.to_dict()["edges"]))
        e2e_s = over_ranks(statistics.median(times), "max", dev)
        h2d = h_off.numel() * h_off.element_size() + h_idx.numel() * 4 + (0 if h_w is None else h_w.numel() * 4)
        out["e2e"] = {"value": over_ranks(statistics.median(edges), "sum", dev) / e2e_s, "unit": "edges/s",
                      "ms_per_step": e2e_s * 1000, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": csr.n * 4 + 8,
                      "includes": "lpa_create from pinned host CSR (copy, validation, buckets), lpa_run, "
                                  "lpa_labels to pinned host, lpa_modularity, lpa_destroy"}
    tuning = g.tuning().to_dict()
    g.close()

    # parity and the CPU baseline (rank 0, one GPU)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        host = dict(machine=platform.machine(), nproc=os.cpu_count(), cpu=_cpu_model())
        if workload == "rmat26":
            # the oracle on a bounded sample of the first sweep; the whole run extrapolated from its rate
            if "rmat26" not in _CPU_SAMPLE:
                _CPU_SAMPLE["rmat26"] = cpu_baseline(csr, target_s=args.ref_seconds)
            cb = dict(_CPU_SAMPLE["rmat26"])
            total_edges = sum(last["edges"])
            cb["full_run_seconds_extrapolated"] = round(total_edges / cb["value"], 1)
            cb["full_run_note"] = ("extrapolated: the GPU run's scanned entries over the sampled single-thread rate "
                                   "(the whole single-thread run would take about that long)")
            out["cpu_baseline"] = cb
            if mode_name == "sync":
                mc, r = cpu_multicore(csr, h_off, h_idx, h_w, full=True)
                out["cpu_multicore"] = mc
                out["parity"] = {"against": "multicore baseline (pinned equal to the oracle's synchronous run), "
                                            "whole graph, whole run",
                                 "labels_equal": bool(torch.equal(labels_gpu, torch.from_numpy(r.labels))),
                                 "dN_equal": r.dN == last["changed"], "edges_equal": r.edges == last["edges"],
                                 "sweeps": r.iterations, "dN_cpu": r.dN}
        else:
            og, r, secs, rw = oracle_full_run(csr, mode_name, tuning if mode_name == "async" else None)
            out["cpu_baseline"] = {"value": sum(r.edges) / secs, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                   "seconds": round(secs, 3), "iterations": r.iterations,
                                   "modularity": oracle.modularity(og, r.labels),
                                   "sample": f"the whole {mode_name} run of the oracle (single-threaded C, "
                                             f"{'sequential id order' if mode_name == 'async' else 'double-buffered'})"
                                             f" on the same graph: {sum(r.edges)} CSR entries scanned",
                                   "host": host}
            if mode_name == "sync":
                out["parity"] = {"against": "oracle synchronous run, whole graph",
                                 "labels_equal": bool(np.array_equal(labels_gpu.numpy(), r.labels)),
                                 "dN_equal": r.dN == last["changed"], "edges_equal": r.edges == last["edges"],
                                 "sweeps": r.iterations}
            else:
                q_w = oracle.modularity(og, rw.labels)
                viol = oracle.violations(og, labels_gpu) / og.n
                q_med = statistics.median(qs)
                out["parity"] = {"against": "oracle asynchronous run under the wave model of the GPU schedule; the "
                                            "GPU's racy result read as the median over the timed runs",
                                 "q_gpu_median": q_med, "q_gpu_min": min(qs), "q_gpu_max": max(qs), "runs": len(qs),
                                 "q_oracle_waves": q_w, "q_oracle_sequential": oracle.modularity(og, r.labels),
                                 "abs_diff_median": abs(q_med - q_w), "within_0_005": abs(q_med - q_w) <= 0.005,
                                 "max_abs_diff": max(abs(x - q_w) for x in qs),
                                 "violation_fraction_last_run": viol,
                                 "violations_within_tolerance": viol <= ALG["tolerance"]}
    return out


def ablations(args, lpa, dev, g, mode):
    """Section 4.2's probe schemes, Section 4.4's value types and Section 4.1's swap
    mitigations on the same resident graph (after the timed region)."""
    res = {}
    ab = {}
    names = {0: "quadratic-double", 1: "linear", 2: "quadratic", 3: "double"}
    for pr in (1, 2, 3, 0):
        g.set_tuning(probe=pr)
        best = None
        for _ in range(2):
            st = g.run(ALG["tolerance"], ALG["max_iters"], ALG["pl_period"], mode).to_dict()
            if best is None or st["total_ms"] < best["total_ms"]:
                best = st
        ab[names[pr]] = {"run_ms": round(best["total_ms"], 2), "probe_fallbacks": best["probe_fallbacks"],
                         "iterations": best["iterations"]}
    res["probe_ablation"] = ab
    va = {}
    for name, fv in (("float64", 2), ("float32", 1), ("uint32", 0)):
        g.set_tuning(float_values=fv)
        best = None
        for _ in range(2):
            st = g.run(ALG["tolerance"], ALG["max_iters"], ALG["pl_period"], mode).to_dict()
            if best is None or st["total_ms"] < best["total_ms"]:
                best = st
        va[name] = {"run_ms": round(best["total_ms"], 2), "iterations": best["iterations"],
                    "modularity": g.modularity(), "device_gb": round(g.device_bytes() / 1e9, 2)}
    res["value_ablation"] = va
    if mode == lpa.SYNC:
        sw = {}
        for name, pl, cc in (("none", 0, 0), ("PL4", 4, 0), ("CC1", 0, 1), ("CC2", 0, 2), ("PL4+CC4", 4, 4),
                             ("PL2+CC2", 2, 2)):
            st = g.run(ALG["tolerance"], ALG["max_iters"], pl, mode, cc_period=cc).to_dict()
            sw[name] = {"run_ms": round(st["total_ms"], 2), "iterations": st["iterations"],
                        "converged": st["converged"], "modularity": g.modularity()}
        res["swap_mitigation"] = {"rmat26": sw, "sbm": swap_sbm(lpa, dev)}
    return res


# the other single-graph configurations, reported beside the headline: (workload, mode, steps)
SIDE_LINES = (("rmat26", "async", 5), ("rmat22", "sync", 10), ("rmat22", "async", 10), ("sbm", "sync", 20),
              ("sbm", "async", 20))


def run_ours(args):
    from paper_2411_11468_gb300 import build, lpa
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    lpa.load()
    line = measure_single(args, lpa, dev, args.workload, args.mode, args.steps, args.warmup, args.e2e_steps,
                          extras=True)
    if ws == 1 and not args.no_extras and args.workload == "rmat26" and args.mode == "sync":
        side = {}
        for wl, md, k in SIDE_LINES:
            torch.cuda.empty_cache()
            side[f"{wl}_{md}"] = measure_single(args, lpa, dev, wl, md, k, max(3, args.warmup), args.e2e_steps)
        line["lines"] = side
    # the batched and served workloads, summarised in the same line (one GPU only)
    if ws == 1 and not args.no_extras:
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        mode = lpa.SYNC if args.mode == "sync" else lpa.ASYNC
        clocks = Clocks(local)
        clocks.start()
        line["batch"] = bench_batch(args, dev, lpa, mode)
        line["serve"] = bench_serve(args, dev, lpa, mode)
        line["clocks_extras"] = clocks.stop()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------------------
# batched and served workloads

def _pinned(t):
    return None if t is None else t.cpu().pin_memory()


def _pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(math.ceil(p / 100.0 * len(xs))) - 1))
    return xs[k]


def bench_batch(args, dev, lpa, mode):
    """4,096 SBM graphs (vertex counts log-uniform in [100, 1e5], block sizes log-uniform in
    [10, 1000], mean degree uniform in [4, 32], unit float32 weights) solved by lpa_batch_run
    (every sweep of every graph in shared launches, replayed from a CUDA graph), against a
    serial loop of lpa_run over the same resident graphs; labels must be identical."""
    from paper_2411_11468_gb300 import graphgen as gg
    t0 = time.time()
    specs = gg.batch_specs(args.batch_graphs)
    graphs = [gg.batch_graph(sp, weights="unit", device=dev) for sp in specs]
    torch.cuda.synchronize()
    n_tot = sum(g.n for g in graphs)
    m_tot = sum(g.m for g in graphs)
    log(f"[bench] batch: {len(graphs)} graphs, {n_tot} vertices, {m_tot} entries, generated in {time.time() - t0:.1f}s")
    b = lpa.Batch([(g.offsets, g.indices, g.weights) for g in graphs])
    run_args = (ALG["tolerance"], ALG["max_iters"], ALG["pl_period"], mode)
    tuned = None
    if not args.no_autotune:
        t1 = time.time()
        default_ms = min(b.run(*run_args)[1] for _ in range(2))
        best, best_ms, count = b.autotune(*run_args, reps=2)
        tuned = {"tuning": best, "device_ms": best_ms, "default_device_ms": default_ms, "configurations": count,
                 "seconds": time.time() - t1}
        log(f"[bench] batch autotune: {default_ms:.1f} -> {best_ms:.1f} ms in {tuned['seconds']:.1f}s ({count} configs)")
    for _ in range(args.warmup):
        res, dms = b.run(*run_args)
    times, dev_ms = [], []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        res, dms = b.run(*run_args)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t1)
        dev_ms.append(dms)
    batch_s = statistics.median(times)
    iters = [r["iterations"] for r in res]
    scanned_bound = sum(g.m * it for g, it in zip(graphs, iters))
    saved = [b.labels(i).clone() for i in range(len(graphs))]
    q = b.modularity()
    # serial loop over the same resident graphs (borrowed handles, one lpa_run each)
    handles = [b.graph(i) for i in range(len(graphs))]
    for h in handles[: min(64, len(handles))]:
        h.run(*run_args)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    serial_iters = [h.run(*run_args).iterations for h in handles]
    torch.cuda.synchronize()
    serial_s = time.perf_counter() - t1
    identical = all(torch.equal(saved[i], b.labels(i)) for i in range(len(graphs))) and serial_iters == iters
    out = {"graphs": len(graphs), "vertices": n_tot, "entries": m_tot,
           "graphs_per_s": len(graphs) / batch_s, "ms_per_step": batch_s * 1000.0,
           "device_ms_per_step": statistics.median(dev_ms),
           "serial_graphs_per_s": len(graphs) / serial_s, "serial_ms": serial_s * 1000.0,
           "speedup_vs_serial": serial_s / batch_s, "identical_labels": bool(identical),
           "iterations_mean": sum(iters) / len(iters), "iterations_max": max(iters),
           "entries_x_iterations_per_s": scanned_bound / batch_s,
           "modularity_mean": sum(q) / len(q), "autotune": tuned,
           "graph_recipe": "SBM, n log-uniform [100, 1e5], block log-uniform [10, 1000], mean degree uniform "
                           "[4, 32] split 8:1 intra:inter, unit float32 weights, seeds 0..count-1"}
    # end to end: pinned host CSR in, labels out, through the public batch API
    if not args.no_e2e:
        host = [(_pinned(g.offsets), _pinned(g.indices), _pinned(g.weights)) for g in graphs]
        labs = [torch.empty(g.n, dtype=torch.int32).pin_memory() for g in graphs]
        del b, handles, saved
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        b2 = lpa.Batch(host)
        b2.run(*run_args)
        for i in range(len(graphs)):
            b2.labels(i, labs[i])
        b2.modularity()
        b2.close()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t1
        h2d = sum(h[0].numel() * h[0].element_size() + h[1].numel() * 4 + (0 if h[2] is None else h[2].numel() * 4)
                  for h in host)
        out["e2e"] = {"value": len(graphs) / e2e_s, "unit": "graphs/s", "ms_per_step": e2e_s * 1000.0,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4 * n_tot + 8 * len(graphs),
                      "includes": "lpa_batch_create from pinned host CSR, lpa_batch_run, lpa_batch_labels to pinned "
                                  "host for every graph, lpa_batch_modularity, lpa_batch_destroy"}
    return out


def bench_serve(args, dev, lpa, mode):
    """A Poisson stream of requests drawn from a pool of seeded SBM / R-MAT graphs with 1e3..1e7
    CSR entries (integer weights 1..8) into lpa_server (continuous batching, admission by HBM
    footprint under the budget); p50/p99 latency from arrival to finish and throughput.  A
    sample of the stream is also run one request at a time (lpa_create, lpa_run, lpa_labels,
    lpa_destroy) and through the server with every request queued at once; the labels of
    both must be identical."""
    from paper_2411_11468_gb300 import graphgen as gg
    import numpy as np
    t0 = time.time()
    specs = gg.serve_specs(args.serve_pool)
    pool = []
    for sp in specs:
        g = gg.serve_graph(sp, device=dev)
        pool.append((_pinned(g.offsets), _pinned(g.indices), _pinned(g.weights)))
        del g
    torch.cuda.synchronize()
    sizes = [p[1].numel() for p in pool]
    log(f"[bench] serve: pool of {len(pool)} graphs, {sum(sizes)} entries, built in {time.time() - t0:.1f}s")
    rng = np.random.default_rng(12345)
    picks = rng.integers(0, len(pool), args.serve_requests)
    budget = int(args.serve_budget_gb * (1 << 30))
    run_args = (ALG["tolerance"], ALG["max_iters"], ALG["pl_period"], mode)

    def drive(req_ids, arrivals):
        """Feeds requests at their arrival times (seconds from start) into a fresh server; returns
        per-request (latency s, iterations, labels or None), wall seconds and server steps."""
        srv = lpa.Server(budget, max_resident=args.serve_resident)
        keep_labels = arrivals is None
        lat, its = {}, {}
        labels = {}
        t_arr = {}
        steps = 0
        i = 0
        total = len(req_ids)
        start = time.perf_counter()
        while len(lat) < total:
            now = time.perf_counter() - start
            while i < total and (arrivals is None or arrivals[i] <= now):
                p = pool[req_ids[i]]
                rid = srv.submit(p[0], p[1], p[2], *run_args, borrow=True)
                t_arr[rid] = (start + (0.0 if arrivals is None else arrivals[i]), i)
                i += 1
            c, running, queued = srv.step()
            steps += 1
            for rid in srv.poll():
                lab, res, _ = srv.result(rid)
                t_done = time.perf_counter()
                ta, k = t_arr.pop(rid)
                lat[k] = t_done - ta
                its[k] = res["iterations"]
                if keep_labels:
                    labels[k] = lab
            if running == 0 and queued == 0 and i < total and arrivals is not None:
                time.sleep(max(0.0, min(0.01, arrivals[i] - (time.perf_counter() - start))))
        wall = time.perf_counter() - start
        srv.close()
        return lat, its, labels, wall, steps

    # one request at a time on a sample, and the same sample through the server at once
    sample = [int(x) for x in picks[: args.serve_sample]]
    for k in sample[:8]:
        gw = lpa.Graph(*pool[k])
        gw.run(*run_args)
        gw.close()
    torch.cuda.synchronize()
    serial_labels = []
    t1 = time.perf_counter()
    for k in sample:
        gs = lpa.Graph(*pool[k])
        gs.run(*run_args)
        serial_labels.append(gs.labels(torch.empty(pool[k][0].numel() - 1, dtype=torch.int32)))
        gs.close()
    torch.cuda.synchronize()
    serial_s = time.perf_counter() - t1
    lat_b, its_b, labels_b, wall_b, steps_b = drive(sample, None)
    identical = all(torch.equal(labels_b[k], serial_labels[k]) for k in range(len(sample)))
    sample_entries = sum(sizes[k] for k in sample)
    # the Poisson stream
    rate = args.serve_rate if args.serve_rate > 0 else 0.7 * len(sample) / wall_b
    arrivals = np.cumsum(rng.exponential(1.0 / rate, args.serve_requests))
    req = [int(x) for x in picks]
    lat, its, _, wall, steps = drive(req, arrivals)
    lats = [lat[k] * 1000.0 for k in range(len(req))]
    entries = sum(sizes[k] for k in req)
    return {"requests": len(req), "rate_per_s": rate, "p50_ms": _pct(lats, 50), "p99_ms": _pct(lats, 99),
            "mean_ms": sum(lats) / len(lats), "wall_s": wall, "requests_per_s": len(req) / wall,
            "entries_per_s": entries / wall,
            "entries_x_iterations_per_s": sum(sizes[k] * its[j] for j, k in enumerate(req)) / wall,
            "server_steps": steps, "budget_gb": args.serve_budget_gb, "max_resident": args.serve_resident,
            "saturated_sample": {"requests": len(sample), "entries": sample_entries,
                                 "server_requests_per_s": len(sample) / wall_b,
                                 "serial_requests_per_s": len(sample) / serial_s,
                                 "speedup_vs_serial": serial_s / wall_b, "identical_labels": bool(identical),
                                 "server_p50_ms": _pct([v * 1000 for v in lat_b.values()], 50),
                                 "server_p99_ms": _pct([v * 1000 for v in lat_b.values()], 99)},
            "pool": {"graphs": len(pool), "entries": sum(sizes),
                     "recipe": "alternating SBM / R-MAT, target entries log-uniform [1e3, 1e7], integer weights "
                               "1..8 as float32; requests pick pool graphs uniformly; latency = finish - arrival"}}


def run_multi(args):
    """--workload batch | serve: one JSON line for the batched or the served workload."""
    from paper_2411_11468_gb300 import build, lpa
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    lpa.load()
    mode = lpa.SYNC if args.mode == "sync" else lpa.ASYNC
    clocks = Clocks(local)
    clocks.start()
    if args.workload == "batch":
        r = bench_batch(args, dev, lpa, mode)
        metric, value, unit, ms = "batched LPA graphs solved per second (4,096 SBM graphs)", r["graphs_per_s"], \
            "graphs/s", r["ms_per_step"]
    else:
        r = bench_serve(args, dev, lpa, mode)
        metric, value, unit, ms = "served LPA requests per second (Poisson stream, continuous batching)", \
            r["requests_per_s"], "requests/s", r["wall_s"] * 1000.0
    clk = clocks.stop()
    line = {"metric": metric, "value": value * ws, "unit": unit, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "mode": args.mode, **ALG}, args.workload: r, "clocks": clk}
    if "e2e" in r:
        line["e2e"] = r["e2e"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch", "serve"], default="rmat26")
    ap.add_argument("--mode", choices=["sync", "async"], default="sync")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and served summaries")
    ap.add_argument("--no-autotune", action="store_true", help="batched workload: keep the default buckets")
    ap.add_argument("--no-ablation", action="store_true", help="skip the probe-scheme and value-type comparisons")
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--serve-requests", type=int, default=20_000)
    ap.add_argument("--serve-pool", type=int, default=512)
    ap.add_argument("--serve-sample", type=int, default=256)
    ap.add_argument("--serve-rate", type=float, default=0.0, help="arrivals/s (0: 70%% of saturated throughput)")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-resident", type=int, default=512)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        log("[bench] warning: fewer than 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch", "serve"):
        return run_multi(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
