"""Wave schedules for `oracle.lpa_async_waves` -- TEST INFRASTRUCTURE.

A model of the order in which the CUDA sweep visits vertices in its asynchronous mode,
written from the launch configuration alone (it holds none of the method's arithmetic and
shares no code with the CUDA path).  The sweep runs one kernel per degree bucket in turn
(thread, lane group, warp, three block tiers, then the hubs).  Inside a bucket, items of
consecutive bucket-list positions go to the resident warps (blocks for the block tiers) in
queue order; a warp fetches 32 vertices of its item at a time and its lane groups take them
32 / G at a time, each group deciding one vertex; a block takes one vertex at a time.  All
hubs are decided together, after every hub's accumulation.  The model lets the resident
warps advance in lockstep: the vertices that all of them decide at the same step form one
wave, which reads the labels as they stand at its start and publishes its moves at its end.
The racy GPU sweep drifts from this lockstep; the model is the schedule the asynchronous
acceptance test compares against.
"""
from __future__ import annotations

import numpy as np

# vertices per work item of the thread, group, warp and block-tier kernels (library defaults)
ITEM_VERTICES = (1024, 256, 64, 16, 8, 4)


def gpu_waves(offsets, tuning: dict, sms: int = 152) -> np.ndarray:
    """wave_of[i] for every vertex of a CSR graph (int64 offsets), for the degree buckets and
    launch shapes in `tuning` (the lpa_tuning fields by name).  Resident warps per SM: 32 for
    the thread, group and warp kernels (their launch bounds); resident blocks per SM for a
    block tier: 2048 / its threads."""
    off = np.asarray(offsets, dtype=np.int64)
    n = off.size - 1
    deg = np.diff(off)
    limits = [tuning["thread_max"], tuning["group_max"], tuning["warp_max"], tuning["cta_max"],
              tuning["cta_large_max"], tuning["cta_xl_max"]]
    threads = [None, None, None, tuning["cta_threads"], tuning["cta_large_threads"], tuning["cta_xl_threads"]]
    lanes = [1, tuning["group_lanes"], 32]
    bucket = np.full(n, -1, dtype=np.int64)           # -1: no entries (never decides)
    lo = 1
    for b, hi in enumerate(limits):
        bucket[(deg >= lo) & (deg <= hi)] = b
        lo = hi + 1
    bucket[deg > limits[-1]] = 6                      # hubs
    wave = np.zeros(n, dtype=np.int64)
    base = 0
    for b in range(6):
        members = np.nonzero(bucket == b)[0]          # ascending ids = bucket-list order
        if members.size == 0:
            continue
        item = tuning.get("item_vertices", 0) if b <= 2 and tuning.get("item_vertices", 0) > 0 else ITEM_VERTICES[b]
        n_items = -(-members.size // item)
        if b <= 2:
            resident = sms * 32
            steps_per_batch = lanes[b] if b > 0 else 1   # 32 / (32 / G) group steps per 32 vertices
        else:
            resident = sms * max(1, 2048 // threads[b])
            steps_per_batch = 32                      # one vertex at a time
        resident = min(resident, n_items)
        batches = -(-item // 32)
        steps_per_item = batches * steps_per_batch
        p = np.arange(members.size, dtype=np.int64)
        k, q = p // item, p % item
        batch, t = q // 32, q % 32
        per_step = 32 // steps_per_batch              # vertices of a batch decided per step
        step = t // per_step
        wave[members] = base + (k // resident) * steps_per_item + batch * steps_per_batch + step
        base = int(wave[members].max()) + 1
    hubs = np.nonzero(bucket == 6)[0]
    if hubs.size:
        wave[hubs] = base
    return wave.astype(np.int32)
