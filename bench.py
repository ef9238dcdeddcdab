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
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
import time

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
    "sbm": dict(kind="sbm", n=10_000, block=100, d_in=16.0, d_out=2.0, weights="unit",
                desc="planted partition 10,000 vertices / 100 blocks, intra-degree 16, inter-degree 2, unit weights"),
}
ALG = dict(tolerance=0.05, max_iters=20, pl_period=4)
BYTES_PER_EDGE_W = 12      # neighbour index 4 + weight 4 + gathered label 4
BYTES_PER_EDGE_U = 8       # unit weights passed as NULL: index 4 + label 4
BYTES_PER_VERTEX = 17      # offsets 2x4 (amortised) + own label 4 + label write 4 + flag 1


def log(*a):
    print(*a, file=sys.stderr, flush=True)


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


def metric_name(workload):
    return f"LPA CSR entries scanned per second, full run to convergence ({workload})"


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
    mode = lpa.SYNC if args.mode == "sync" else lpa.ASYNC
    t0 = time.time()
    csr = make_graph(args.workload, dev)
    torch.cuda.synchronize()
    log(f"[bench] graph {args.workload}: n={csr.n} m={csr.m} generated in {time.time() - t0:.1f}s")
    weighted = csr.weights is not None
    stream = torch.cuda.current_stream(dev)
    g = lpa.Graph(csr.offsets, csr.indices, csr.weights)
    log(f"[bench] lpa_create done; device bytes {g.device_bytes() / 1e9:.2f} GB")

    def step(time_kernels=False):
        st = g.run(ALG["tolerance"], ALG["max_iters"], ALG["pl_period"], mode, time_kernels=time_kernels)
        q = g.modularity()
        return st, q

    for _ in range(args.warmup):
        st, q = step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        st, q = step(time_kernels=True)
        stats.append(st.to_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    edges_per_step = statistics.median(sum(s["edges"]) for s in stats)
    value = ws * edges_per_step / (ms / 1000.0)

    # roofline of the dominant kernel over the timed steps
    peak, peak_src = measured_peaks()
    kms = [0.0] * lpa.NUM_KERNELS
    kbytes = [0.0] * lpa.NUM_KERNELS
    klaunch = [0] * lpa.NUM_KERNELS
    for s in stats:
        kb = kernel_bytes(s, weighted)
        for it in range(len(s["kernel_ms"])):
            for k in range(lpa.NUM_KERNELS):
                if s["kernel_ms"][it][k] > 0:
                    kms[k] += s["kernel_ms"][it][k]
                    klaunch[k] += 1
        for k in range(lpa.NUM_KERNELS):
            kbytes[k] += kb[k]
    # hub accumulate owns the hub edges; its bytes are the scanned-entry bytes
    dom = max(range(lpa.NUM_KERNELS), key=lambda k: kms[k])
    achieved = kbytes[dom] / (kms[dom] / 1000.0) / 1e9 if kms[dom] > 0 else 0.0
    first = stats[-1]
    sweep0_ms = first["iter_ms"][0]
    sweep0_bytes = (BYTES_PER_EDGE_W if weighted else BYTES_PER_EDGE_U) * first["edges"][0] + \
        BYTES_PER_VERTEX * first["active"][0]
    kernel_table = {lpa.KERNEL_NAMES[k]: dict(ms_per_step=round(kms[k] / args.steps, 4), launches_per_step=klaunch[k] / args.steps,
                                              gbs=round(kbytes[k] / (kms[k] / 1000.0) / 1e9, 1) if kms[k] > 0 else None)
                    for k in range(lpa.NUM_KERNELS) if kms[k] > 0}
    roofline = {"bound": "hbm", "kernel": lpa.KERNEL_NAMES[dom], "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None, "peak_source": peak_src,
                "bytes_model": f"{BYTES_PER_EDGE_W if weighted else BYTES_PER_EDGE_U} B per scanned entry + "
                               f"{BYTES_PER_VERTEX} B per processed vertex",
                "first_sweep": {"ms": round(sweep0_ms, 3), "edges": first["edges"][0],
                                "edges_per_s": first["edges"][0] / (sweep0_ms / 1000.0),
                                "gbs": round(sweep0_bytes / (sweep0_ms / 1000.0) / 1e9, 1),
                                "frac": round(sweep0_bytes / (sweep0_ms / 1000.0) / 1e9 / peak, 4)},
                "kernels": kernel_table}

    line = {"metric": metric_name(args.workload), "value": value, "unit": "edges/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "graph": WORKLOADS[args.workload]["desc"], "n": csr.n, "m": csr.m,
                       "mode": args.mode, **ALG, "l2": "inputs larger than L2 (CSR resident in HBM)"},
            "iterations": first["iterations"], "dN": first["changed"], "edges_per_sweep": first["edges"],
            "modularity": q, "processing_rate": ws * csr.m / (ms / 1000.0),
            "roofline": roofline, "gpu_launches": int(statistics.median(s["launches"] for s in stats)) + 2,
            "clocks": clk, "probe_fallbacks": first["probe_fallbacks"],
            "sweeps": [{"ms": round(first["iter_ms"][i], 3), "edges": first["edges"][i], "active": first["active"][i],
                        "changed": first["changed"][i],
                        "kernels": {lpa.KERNEL_NAMES[k]: [round(first["kernel_ms"][i][k], 3), first["kernel_active"][i][k],
                                                          first["kernel_edges"][i][k]]
                                    for k in range(lpa.NUM_KERNELS) if first["kernel_ms"][i][k] > 0}}
                       for i in range(len(first["iter_ms"]))]}

    # end to end through the public API with host buffers
    if not args.no_e2e:
        h_off = csr.offsets.cpu().pin_memory()
        h_idx = csr.indices.cpu().pin_memory()
        h_w = None if csr.weights is None else csr.weights.cpu().pin_memory()
        h_lab = torch.empty(csr.n, dtype=torch.int32).pin_memory()
        del g
        torch.cuda.synchronize()
        times = []
        edges = []
        for rep in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g2 = lpa.Graph(h_off, h_idx, h_w)
            st2 = g2.run(ALG["tolerance"], ALG["max_iters"], ALG["pl_period"], mode)
            g2.labels(h_lab)
            q2 = g2.modularity()
            g2.close()
            torch.cuda.synchronize()
            if rep > 0:
                times.append(time.perf_counter() - t0)
                edges.append(sum(st2.to_dict()["edges"]))
        e2e_s = statistics.median(times)
        if ws > 1:
            t = torch.tensor([e2e_s], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = h_off.numel() * h_off.element_size() + h_idx.numel() * 4 + (0 if h_w is None else h_w.numel() * 4)
        line["e2e"] = {"value": ws * statistics.median(edges) / e2e_s, "unit": "edges/s", "ms_per_step": e2e_s * 1000,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": csr.n * 4 + 8,
                       "includes": "lpa_create from pinned host CSR (copy, validation, buckets), lpa_run, "
                                   "lpa_labels to pinned host, lpa_modularity, lpa_destroy"}
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(csr, target_s=args.ref_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat26")
    ap.add_argument("--mode", choices=["sync", "async"], default="sync")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        log("[bench] warning: fewer than 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
