"""Wave schedules for `oracle.lpa_async_waves` -- TEST INFRASTRUCTURE.

A model of the order in which the CUDA sweep visits vertices in its asynchronous mode,
written from the launch configuration alone (it holds none of the method's arithmetic and
shares no code with the CUDA path).  The sweep runs one kernel per degree bucket in turn
(thread, lane group, warp, three block tiers, then the hubs), each over the bucket's vertex
list in id order, cut into work items that warps (blocks, for the block tiers) take from a
queue.

  * Thread, group and warp buckets, per-vertex kernels: a warp takes 32 list positions of its
    item at a time and its 32 / G lane groups (G = 1, group_lanes, 32) decide one vertex each
    per step.  Resident: 32 warps per SM.
  * The same buckets when their bit of flat_buckets is set (flattened kernel): a warp takes 32
    list positions at a time and packs them, in order, into sub-batches whose tables (2^b
    slots each, 2^b - 1 >= D << shift) fit its shared-memory region (at least 1,024 slots,
    more when the bucket's largest table needs it); a sub-batch reads its neighbours' labels
    and then decides all its vertices together: one step.  Resident: 24 warps per SM.
  * Block tiers: a block decides one vertex per step.
  * Hubs: every hub's accumulation ends before any hub decides: one step.

The model lets every resident warp (block) advance one step per time unit, taking the next
item from the queue when its item is done; the vertices decided at the same time form one
wave, which reads the labels as they stand at its start and publishes its moves at its end.
Every kernel takes the processed flags of a 32-vertex batch when it fetches the batch, before
its first step on it: that is each vertex's take wave (`take_of`).
The racy GPU sweep drifts from this lockstep; the model is the schedule the asynchronous
acceptance test compares against.
"""
from __future__ import annotations

import heapq

import numpy as np

# vertices per work item of the thread, group, warp and block-tier kernels (library defaults)
ITEM_VERTICES = (1024, 256, 64, 16, 8, 4)
FLAT_MIN_SLOTS = 1024          # table slots of a warp region, at least
FLAT_WARPS_PER_SM = 24         # resident warps of the flattened kernel per SM (3 blocks of 8)
GROUP_WARPS_PER_SM = 32        # resident warps of the per-vertex thread / group / warp kernels


def _cap_bits(x: np.ndarray) -> np.ndarray:
    """Smallest b with 2^b - 1 >= x (x >= 1)."""
    return np.floor(np.log2(x.astype(np.float64))).astype(np.int64) + 1


def _schedule(durations, resident):
    """Start time of each item when `resident` workers take items in queue order."""
    free = [0] * max(1, min(resident, len(durations)))
    heapq.heapify(free)
    starts = np.zeros(len(durations), dtype=np.int64)
    for k, d in enumerate(durations):
        t = heapq.heappop(free)
        starts[k] = t
        heapq.heappush(free, t + int(d))
    return starts


def gpu_waves(offsets, tuning: dict, sms: int = 152) -> np.ndarray:
    """wave_of[i] (the deciding wave) for every vertex of a CSR graph (int64 offsets)."""
    return gpu_schedule(offsets, tuning, sms)[0]


def gpu_schedule(offsets, tuning: dict, sms: int = 152):
    """(wave_of, take_of) for every vertex of a CSR graph (int64 offsets), for the degree
    buckets and launch shapes in `tuning` (the lpa_tuning fields by name): the wave in which
    each vertex decides and the wave in which its batch's flags are taken."""
    off = np.asarray(offsets, dtype=np.int64)
    n = off.size - 1
    deg = np.diff(off)
    shift = int(tuning.get("smem_table_shift", 1))
    limits = [tuning["thread_max"], tuning["group_max"], tuning["warp_max"], tuning["cta_max"],
              tuning["cta_large_max"], tuning["cta_xl_max"]]
    threads = [None, None, None, tuning["cta_threads"], tuning["cta_large_threads"], tuning["cta_xl_threads"]]
    bucket = np.full(n, -1, dtype=np.int64)           # -1: no entries (never decides)
    lo = 1
    for b, hi in enumerate(limits):
        bucket[(deg >= lo) & (deg <= hi)] = b
        lo = hi + 1
    bucket[deg > limits[-1]] = 6                      # hubs
    wave = np.zeros(n, dtype=np.int64)
    take = np.zeros(n, dtype=np.int64)
    base = 0
    for b in range(6):
        members = np.nonzero(bucket == b)[0]          # ascending ids = bucket-list order
        if members.size == 0:
            continue
        iv = int(tuning.get("item_vertices", 0) or 0)
        item = iv if (b <= 2 and iv > 0) else ITEM_VERTICES[b]
        n_items = -(-members.size // item)
        step = np.zeros(members.size, dtype=np.int64)     # step within the item
        dur = np.zeros(n_items, dtype=np.int64)
        flat = bool((int(tuning.get("flat_buckets", 0)) >> b) & 1) if b <= 2 else False
        if b <= 2 and not flat:
            lanes = (1, int(tuning["group_lanes"]), 32)[b]
            per_step = 32 // lanes                    # vertices of a 32-vertex batch decided per step
            p = np.arange(members.size, dtype=np.int64)
            q = p % item
            step[:] = (q // 32) * lanes + (q % 32) // per_step
            dur[:] = -(-item // 32) * lanes
            resident = sms * GROUP_WARPS_PER_SM
        elif b <= 2:
            region = max(FLAT_MIN_SLOTS, 1 << int(_cap_bits(np.array([max(limits[b], 1) << shift]))[0]))
            caps = 1 << _cap_bits(deg[members] << shift)
            for k in range(n_items):
                s = 0
                for c0 in range(k * item, min((k + 1) * item, members.size), 32):
                    used = 0
                    for p in range(c0, min(c0 + 32, (k + 1) * item, members.size)):
                        if used + caps[p] > region:
                            s += 1
                            used = 0
                        used += caps[p]
                        step[p] = s
                    s += 1
                dur[k] = s
            resident = sms * FLAT_WARPS_PER_SM
        else:
            p = np.arange(members.size, dtype=np.int64)
            step[:] = p % item
            dur[:] = item
            dur[-1] = members.size - (n_items - 1) * item
            resident = sms * max(1, 2048 // threads[b])
        starts = _schedule(dur, resident)
        p = np.arange(members.size, dtype=np.int64)
        k_of = p // item
        wave[members] = base + starts[k_of] + step
        first = k_of * item + ((p % item) // 32) * 32          # first position of the vertex's batch
        take[members] = base + starts[k_of] + step[first]
        base = int(wave[members].max()) + 1
    hubs = np.nonzero(bucket == 6)[0]
    if hubs.size:
        wave[hubs] = base
        take[hubs] = base
    return wave.astype(np.int32), take.astype(np.int32)
