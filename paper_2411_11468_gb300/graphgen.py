"""Seeded synthetic graph generators (inputs only; no label-propagation arithmetic).

This module is the one piece shared by the CPU oracle tests and the CUDA path: it
produces undirected weighted graphs in CSR form (int64 offsets, int32 neighbour
indices, float32 weights), the input format of the paper's Preliminaries section
(graph G(V, E, w) with w_ij = w_ji, reverse edges added, unit weights by default).

Every random draw is counter based: value(seed, stream, ctr) = mix(key(seed, stream)
+ (ctr + 1) * GOLDEN) with the SplitMix64 finaliser (Steele, Lea and Flood, 2014),
written with torch int64 tensors (two's-complement wraparound, logical shifts
emulated by masking).  Only integer arithmetic decides the graph, so the same call
gives the same CSR on the CPU and on a CUDA device.

Generators:
  * rmat()  -- R-MAT (Chakrabarti, Zhan, Faloutsos 2004), symmetrised, self-loops
               and duplicates removed; unit weights or integer weights in [1, 8].
  * sbm()   -- planted partition with equal contiguous blocks, edges drawn by
               counter-based edge sampling (intra and inter draws), duplicates merged.
  * small closed-form graphs used as test fixtures (cliques, bridge, K_{n,n}, star).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import torch

GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

# stream ids keep independent draws apart
STREAM_RMAT = 1
STREAM_WEIGHT = 2
STREAM_SBM_IN_U = 3
STREAM_SBM_IN_V = 4
STREAM_SBM_OUT_U = 5
STREAM_SBM_OUT_V = 6
STREAM_BATCH = 7
STREAM_SERVE = 8


def _s64(x: int) -> int:
    """Python int in [0, 2^64) -> the int64 with the same bits."""
    x &= MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def _lsr(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def mix64(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function on int64 bit patterns (wraparound multiply)."""
    z = (z ^ _lsr(z, 30)) * _s64(MIX1)
    z = (z ^ _lsr(z, 27)) * _s64(MIX2)
    return z ^ _lsr(z, 31)


def mix64_int(z: int) -> int:
    """Same function on a Python int (used for keys and for pinning the tensor version)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return mix64_int(mix64_int(seed * GOLDEN + stream) + stream)


def draws(seed: int, stream: int, ctr: torch.Tensor) -> torch.Tensor:
    """64-bit pseudo-random bit patterns (int64) for integer counters `ctr`."""
    key = _s64(stream_key(seed, stream))
    return mix64(key + (ctr + 1) * _s64(GOLDEN))


def draws53(seed: int, stream: int, ctr: torch.Tensor) -> torch.Tensor:
    """Non-negative 53-bit integers (uniform in [0, 2^53))."""
    return _lsr(draws(seed, stream, ctr), 11)


@dataclass
class CSRGraph:
    """Undirected graph in CSR form; every edge is stored in both directions."""
    offsets: torch.Tensor          # int64 [n+1]
    indices: torch.Tensor          # int32 [m]
    weights: Optional[torch.Tensor]  # float32 [m] or None (unit)
    name: str = ""
    planted: Optional[torch.Tensor] = None  # int32 [n] planted block id (SBM)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.offsets.numel() - 1

    @property
    def m(self) -> int:
        return self.indices.numel()

    def to(self, device) -> "CSRGraph":
        return CSRGraph(self.offsets.to(device), self.indices.to(device),
                        None if self.weights is None else self.weights.to(device),
                        self.name, None if self.planted is None else self.planted.to(device),
                        dict(self.meta))

    def degrees(self) -> torch.Tensor:
        return self.offsets[1:] - self.offsets[:-1]


def csr_from_directed_keys(keys: torch.Tensor, n: int) -> tuple[torch.Tensor, torch.Tensor]:
    """Sorted, unique int64 keys u*n+v -> (offsets int64, indices int32)."""
    u = keys // n
    v = keys - u * n
    deg = torch.bincount(u, minlength=n)
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=keys.device)
    torch.cumsum(deg, 0, out=offsets[1:])
    return offsets, v.to(torch.int32)


def _symmetrise_unique(u: torch.Tensor, v: torch.Tensor, n: int) -> torch.Tensor:
    keep = u != v
    u, v = u[keep], v[keep]
    keys = torch.cat([u * n + v, v * n + u])
    keys = torch.unique(keys, sorted=True)
    return keys


def edge_weights(seed: int, offsets: torch.Tensor, indices: torch.Tensor,
                 kind: str, chunk: int = 1 << 27) -> Optional[torch.Tensor]:
    """Per-entry float32 weights; both directions of an edge get the same value.

    kind: "unit" -> all 1.0 (float32 array), "none" -> None (caller passes no weights),
          "int8" -> 1 + (hash(min(u,v), max(u,v)) mod 8), an integer in [1, 8].
    """
    m = indices.numel()
    n = offsets.numel() - 1
    if kind == "none":
        return None
    if kind == "unit":
        return torch.ones(m, dtype=torch.float32, device=indices.device)
    if kind != "int8":
        raise ValueError(f"unknown weight kind {kind!r}")
    out = torch.empty(m, dtype=torch.float32, device=indices.device)
    deg = offsets[1:] - offsets[:-1]
    # walk rows in chunks of roughly `chunk` entries
    v0 = 0
    while v0 < n:
        e0 = int(offsets[v0])
        target = e0 + chunk
        v1 = int(torch.searchsorted(offsets, torch.tensor([target], device=offsets.device,
                                                          dtype=torch.int64), right=True)[0]) - 1
        v1 = max(v1, v0 + 1)
        v1 = min(v1, n)
        e1 = int(offsets[v1])
        if e1 > e0:
            u = torch.repeat_interleave(torch.arange(v0, v1, device=indices.device, dtype=torch.int64),
                                        deg[v0:v1])
            w = indices[e0:e1].to(torch.int64)
            lo = torch.minimum(u, w)
            hi = torch.maximum(u, w)
            h = draws(seed, STREAM_WEIGHT, lo * n + hi)
            out[e0:e1] = (1 + (_lsr(h, 20) & 7)).to(torch.float32)
        v0 = v1
    return out


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, weights: str = "unit", device="cpu", chunk_edges: int = 1 << 25) -> CSRGraph:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale generated edges.

    Each generated edge descends `scale` levels of the adjacency matrix; at level l the
    quadrant is chosen by comparing a 53-bit draw with floor(a*2^53), floor((a+b)*2^53),
    floor((a+b+c)*2^53) (most significant bit first, no noise, no permutation, so
    vertex 0 is the largest hub).  The edge list is then symmetrised and self-loops
    and duplicates are removed.
    """
    n = 1 << scale
    m0 = edge_factor * n
    t_a = int(a * (1 << 53))
    t_ab = int((a + b) * (1 << 53))
    t_abc = int((a + b + c) * (1 << 53))
    dev = torch.device(device)
    keys_all = torch.empty(2 * m0, dtype=torch.int64, device=dev)
    fill = 0
    for e0 in range(0, m0, chunk_edges):
        e1 = min(m0, e0 + chunk_edges)
        e = torch.arange(e0, e1, dtype=torch.int64, device=dev)
        u = torch.zeros_like(e)
        v = torch.zeros_like(e)
        base = e * 64
        for lvl in range(scale):
            r = draws53(seed, STREAM_RMAT, base + lvl)
            bu = (r >= t_ab).to(torch.int64)                      # quadrants c, d -> lower half
            bv = ((r >= t_a) & (r < t_ab)) | (r >= t_abc)         # quadrants b, d -> right half
            u = u * 2 + bu
            v = v * 2 + bv.to(torch.int64)
        keep = u != v
        u, v = u[keep], v[keep]
        k = u.numel()
        keys_all[fill:fill + k] = u * n + v
        keys_all[fill + k:fill + 2 * k] = v * n + u
        fill += 2 * k
        del e, u, v, base
    keys_all = keys_all[:fill]
    # sort + dedupe in partitions of the source-vertex range (top bits of u)
    pbits = max(0, min(6, scale - 10))
    parts = []
    degs = torch.zeros(n, dtype=torch.int64, device=dev)
    shift = scale + (scale - pbits)  # key = u*n + v ; u's top pbits are key >> shift
    for p in range(1 << pbits):
        if pbits:
            sel = keys_all[_lsr(keys_all, shift) == p]
        else:
            sel = keys_all
        sel = torch.unique(sel, sorted=True)
        uu = sel >> scale
        degs += torch.bincount(uu, minlength=n)
        parts.append((sel & (n - 1)).to(torch.int32))
        del sel, uu
    del keys_all
    indices = torch.cat(parts) if len(parts) > 1 else parts[0]
    del parts
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(degs, 0, out=offsets[1:])
    w = edge_weights(seed, offsets, indices, weights)
    return CSRGraph(offsets, indices, w, name=f"rmat{scale}",
                    meta=dict(scale=scale, edge_factor=edge_factor, a=a, b=b, c=c, seed=seed,
                              weights=weights))


def _draw_count(target: float, pairs: int) -> int:
    """Number of uniform draws (with replacement) whose expected count of distinct pairs is
    `target` among `pairs` equally likely pairs: pairs * (1 - (1 - 1/pairs)^d) = target."""
    if pairs <= 0 or target <= 0:
        return 0
    if pairs == 1:
        return 8
    if target >= pairs * 0.999:
        return int(8 * pairs)
    return int(math.ceil(math.log(1.0 - target / pairs) / math.log(1.0 - 1.0 / pairs)))


def sbm(n: int, block: int, d_in: float, d_out: float, seed: int = 0, weights: str = "unit",
        device="cpu", stream_offset: int = 0) -> CSRGraph:
    """Planted partition: contiguous blocks of `block` vertices (the last may be smaller).

    Intra-block edges: draws of (u uniform, v uniform among the other members of u's
    block), as many as make the expected number of distinct intra pairs n*d_in/2.
    Inter-block edges: n*d_out/2 draws of (u uniform, v uniform outside u's block).
    Both directions are stored and duplicate pairs merged, so the expected
    intra-degree is d_in (up to the block-size saturation) and the inter-degree ~d_out.
    """
    dev = torch.device(device)
    nb = (n + block - 1) // block
    last = n - (nb - 1) * block
    pairs_in = (nb - 1) * block * (block - 1) // 2 + last * (last - 1) // 2
    d_in_count = _draw_count(n * d_in / 2.0, pairs_in)
    d_out_count = int(round(n * d_out / 2.0)) if nb > 1 else 0
    so = stream_offset * 16
    us, vs = [], []
    if d_in_count:
        ctr = torch.arange(d_in_count, dtype=torch.int64, device=dev)
        u = draws53(seed, STREAM_SBM_IN_U + so, ctr) % n
        bs = (u // block) * block
        sb = torch.clamp(n - bs, max=block)
        ok = sb > 1
        off = draws53(seed, STREAM_SBM_IN_V + so, ctr) % torch.clamp(sb - 1, min=1)
        v = bs + (u - bs + 1 + off) % sb
        us.append(u[ok]); vs.append(v[ok])
    if d_out_count:
        ctr = torch.arange(d_out_count, dtype=torch.int64, device=dev)
        u = draws53(seed, STREAM_SBM_OUT_U + so, ctr) % n
        bs = (u // block) * block
        sb = torch.clamp(n - bs, max=block)
        r = draws53(seed, STREAM_SBM_OUT_V + so, ctr) % (n - sb)
        v = torch.where(r < bs, r, r + sb)
        us.append(u); vs.append(v)
    if us:
        keys = _symmetrise_unique(torch.cat(us), torch.cat(vs), n)
    else:
        keys = torch.empty(0, dtype=torch.int64, device=dev)
    offsets, indices = csr_from_directed_keys(keys, n)
    w = edge_weights(seed + 0x5B5B * (stream_offset + 1), offsets, indices, weights)
    planted = (torch.arange(n, device=dev) // block).to(torch.int32)
    return CSRGraph(offsets, indices, w, name=f"sbm{n}", planted=planted,
                    meta=dict(n=n, block=block, d_in=d_in, d_out=d_out, seed=seed, weights=weights))


def batch_specs(count: int = 4096, seed: int = 0, n_lo: int = 100, n_hi: int = 100_000,
                s_lo: int = 10, s_hi: int = 1000, d_lo: float = 4.0, d_hi: float = 32.0):
    """Per-graph parameters of the batched workload: vertex count and block size
    log-uniform, mean degree uniform, split 8:1 between intra and inter edges."""
    ctr = torch.arange(count, dtype=torch.int64) * 4
    r = draws53(seed, STREAM_BATCH, torch.stack([ctr, ctr + 1, ctr + 2], 1)).to(torch.float64) / float(1 << 53)
    specs = []
    for g in range(count):
        n = int(round(math.exp(math.log(n_lo) + r[g, 0].item() * (math.log(n_hi) - math.log(n_lo)))))
        s = int(round(math.exp(math.log(s_lo) + r[g, 1].item() * (math.log(s_hi) - math.log(s_lo)))))
        s = max(2, min(s, n))
        d = d_lo + r[g, 2].item() * (d_hi - d_lo)
        specs.append(dict(n=n, block=s, d_in=d * 8.0 / 9.0, d_out=d / 9.0, seed=seed + g))
    return specs


def batch_graph(spec: dict, weights: str = "unit", device="cpu") -> CSRGraph:
    return sbm(spec["n"], spec["block"], spec["d_in"], spec["d_out"], seed=spec["seed"],
               weights=weights, device=device)


def serve_specs(count: int = 512, seed: int = 0, e_lo: float = 1e3, e_hi: float = 1e7):
    """Request graphs of the serving workload: half SBM, half R-MAT (alternating), each with a
    target of directed CSR entries log-uniform in [e_lo, e_hi] and integer weights 1..8.

    R-MAT: the smallest scale whose edge factor (target / 2^(scale+1)) is at most 32 (scale at
    least 5).  SBM: mean degree uniform in [4, 32] split 8:1 intra:inter, block size
    log-uniform in [10, 1000].  Duplicate removal makes the realised counts somewhat lower."""
    ctr = torch.arange(count, dtype=torch.int64) * 4
    r = draws53(seed, STREAM_SERVE, torch.stack([ctr, ctr + 1, ctr + 2], 1)).to(torch.float64) / float(1 << 53)
    specs = []
    for k in range(count):
        e = math.exp(math.log(e_lo) + r[k, 0].item() * (math.log(e_hi) - math.log(e_lo)))
        if k % 2 == 0:
            d = 4.0 + r[k, 1].item() * 28.0
            n = max(16, int(round(e / d)))
            s = int(round(math.exp(math.log(10) + r[k, 2].item() * (math.log(1000) - math.log(10)))))
            specs.append(dict(kind="sbm", n=n, block=max(2, min(s, n)), d_in=d * 8.0 / 9.0, d_out=d / 9.0,
                              seed=seed * 1_000_003 + k, target_entries=e))
        else:
            scale = 5
            while e / float(1 << (scale + 1)) > 32.0:
                scale += 1
            ef = max(1, int(round(e / float(1 << (scale + 1)))))
            specs.append(dict(kind="rmat", scale=scale, edge_factor=ef, seed=seed * 1_000_003 + k, target_entries=e))
    return specs


def serve_graph(spec: dict, device="cpu") -> CSRGraph:
    if spec["kind"] == "sbm":
        return sbm(spec["n"], spec["block"], spec["d_in"], spec["d_out"], seed=spec["seed"], weights="int8",
                   device=device)
    return rmat(spec["scale"], edge_factor=spec["edge_factor"], seed=spec["seed"], weights="int8", device=device)


# ----------------------------------------------------------------------------------------
# small closed-form fixtures

def from_edges(n: int, edges, weights=None, symmetric: bool = True, device="cpu") -> CSRGraph:
    """CSR from an undirected edge list [(u, v), ...] (both directions stored, rows sorted).
    weights: optional list aligned with `edges` (same weight in both directions)."""
    es = []
    for k, (u, v) in enumerate(edges):
        w = 1.0 if weights is None else float(weights[k])
        es.append((u, v, w))
        if symmetric and u != v:
            es.append((v, u, w))
    es.sort()
    offsets = torch.zeros(n + 1, dtype=torch.int64)
    for u, _, _ in es:
        offsets[u + 1] += 1
    offsets = torch.cumsum(offsets, 0)
    indices = torch.tensor([v for _, v, _ in es], dtype=torch.int32)
    w = torch.tensor([w for _, _, w in es], dtype=torch.float32)
    g = CSRGraph(offsets, indices, w, name="edges")
    return g.to(device)


def cliques(k: int, s: int) -> CSRGraph:
    """k disjoint cliques K_s with contiguous ids."""
    edges = [(c * s + a, c * s + b) for c in range(k) for a in range(s) for b in range(a + 1, s)]
    return from_edges(k * s, edges)


def two_cliques_bridge(s: int) -> CSRGraph:
    """K_s on [0, s) and K_s on [s, 2s), joined by the edge (s-1, s)."""
    edges = [(a, b) for a in range(s) for b in range(a + 1, s)]
    edges += [(s + a, s + b) for a in range(s) for b in range(a + 1, s)]
    edges.append((s - 1, s))
    return from_edges(2 * s, edges)


def complete_bipartite(n: int) -> CSRGraph:
    """K_{n,n} with sides A = [0, n) and B = [n, 2n)."""
    return from_edges(2 * n, [(a, n + b) for a in range(n) for b in range(n)])


def star(n: int) -> CSRGraph:
    """K_{1,n}: centre 0, leaves 1..n."""
    return from_edges(n + 1, [(0, j) for j in range(1, n + 1)])


def random_small(n: int, p: float, seed: int, wmax: int = 8, self_loops: bool = False) -> CSRGraph:
    """Dense-sampled small graph with integer weights in [1, wmax] (tests; n <= a few hundred)."""
    iu = torch.triu_indices(n, n, 0 if self_loops else 1)
    ctr = iu[0].to(torch.int64) * n + iu[1].to(torch.int64)
    keep = draws53(seed, 11, ctr) < int(p * (1 << 53))
    u, v = iu[0][keep].tolist(), iu[1][keep].tolist()
    w = (1 + draws53(seed, 12, ctr[keep]) % wmax).tolist()
    return from_edges(n, list(zip(u, v)), w)
