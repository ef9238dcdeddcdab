"""The benchmark's roofline bookkeeping (no GPU): algorithmic bytes per kernel slot, and the
DRAM-traffic record that is reported only while the sources it was captured on are unchanged."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2411_11468_gb300 import lpa  # noqa: E402


def _stats(edges, active):
    return {"kernel_edges": edges, "kernel_active": active}


def test_kernel_bytes_counts_entries_and_vertices_per_slot():
    K = lpa.NUM_KERNELS
    edges = [[0] * K for _ in range(2)]
    active = [[0] * K for _ in range(2)]
    edges[0][2], active[0][2] = 1000, 10          # sweep 0, warp slot
    edges[1][2], active[1][2] = 500, 4            # sweep 1, same slot
    edges[1][K - 1], active[1][K - 1] = 7, 1      # another slot
    w = bench.kernel_bytes(_stats(edges, active), weighted=True)
    u = bench.kernel_bytes(_stats(edges, active), weighted=False)
    assert w[2] == 12 * 1500 + 17 * 14 and u[2] == 8 * 1500 + 17 * 14
    assert w[K - 1] == 12 * 7 + 17 and u[K - 1] == 8 * 7 + 17
    assert sum(1 for x in w if x) == 2


def test_traffic_is_a_scaled_rate_reported_only_while_sources_match(monkeypatch):
    csrc = os.path.join(ROOT, "paper_2411_11468_gb300", "csrc")
    name = "lpa_internal.h"
    digest = hashlib.sha256(open(os.path.join(csrc, name), "rb").read()).hexdigest()
    rec = {"captured_on": "rmat22u", "bytes_per_entry": {"hub_acc": 13.5, "warp": 7.0}, "sources": {name: digest}}
    monkeypatch.setattr(bench, "TRAFFIC", rec)
    assert bench.traffic_for("hub_acc", 1e6) == 13.5e6
    assert bench.traffic_for("warp", 2e6) == 14e6
    assert bench.traffic_for("cta", 1e6) is None                     # no rate captured for the slot
    monkeypatch.setattr(bench, "TRAFFIC", dict(rec, sources={name: "0" * 64}))
    assert bench.traffic_for("hub_acc", 1e6) is None                 # source changed since the capture
    monkeypatch.setattr(bench, "TRAFFIC", dict(rec, sources={"no_such_file.cu": digest}))
    assert bench.traffic_for("hub_acc", 1e6) is None
