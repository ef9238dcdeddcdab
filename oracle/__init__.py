"""CPU oracle for nu-LPA label propagation (arXiv 2411.11468) -- TEST INFRASTRUCTURE.

Only the test suite, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the CUDA path (`paper_2411_11468_gb300`)
and never imports it.  The arithmetic lives in `lpa_oracle.c` (plain single-threaded
C11, built with gcc by `build()`); this module only marshals numpy arrays.

Functions and the passages they follow:
  lpa_sync / lpa_async  -- Algorithm 1 (lpa, lpaMove), Eq. 3, Section 4 items (1)-(5)
  lpa_async_waves       -- the asynchronous mode under a schedule of parallel waves (a
                           reading of Section 4 item 1): between lpa_async and lpa_sync
  cross_check           -- Section 4.1's Cross-Check (reverts of bad moves), in id order
  label_weights         -- Preliminaries, K_{i->c}, by sort-and-count
  ht_build / ht_probe_slot / ht_capacity -- Section 4.2 per-vertex hashtable, Algorithm 2
  modularity / modularity_exact          -- Eq. 1 (community form)
  violations            -- vertices whose label is not a max-weight neighbour label
  sweep_range           -- one all-active synchronous sweep over a vertex range
  multicore_lpa_sync    -- the synchronous run on all host cores (OpenMP, lpa_multicore.c):
                           a timing baseline that must give lpa_sync's result
"""
from __future__ import annotations

import ctypes as ct
import os
import platform
import subprocess
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpa_oracle.c")
_LIB = os.path.join(_HERE, f"liblpa_oracle.{platform.machine()}.so")   # per host architecture

MAX_RETRIES = 32      # hashtable probe budget before the linear fallback (reading of Algorithm 2)


_MC_SRC = os.path.join(_HERE, "lpa_multicore.c")
_MC_LIB = os.path.join(_HERE, f"liblpa_multicore.{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, C11), and the multicore baseline with -fopenmp.
    Returns the oracle library path."""
    for src, out, extra in ((_SRC, _LIB, []), (_MC_SRC, _MC_LIB, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
            tmp = out + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", *extra, "-o", tmp, src])
            os.replace(tmp, out)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ct.CDLL(_LIB)
        P = ct.c_void_p
        i64, i32, u32, dbl = ct.c_int64, ct.c_int32, ct.c_uint32, ct.c_double
        L.orc_lpa_sync.argtypes = [i64, P, P, P, dbl, ct.c_int, ct.c_int, ct.c_int, P, P, P, P, P, P]
        L.orc_lpa_sync.restype = ct.c_int
        L.orc_lpa_sync_cc.argtypes = [i64, P, P, P, dbl, ct.c_int, ct.c_int, ct.c_int, ct.c_int, P, P, P, P, P, P]
        L.orc_lpa_sync_cc.restype = ct.c_int
        L.orc_cross_check.argtypes = [i64, P, P]
        L.orc_cross_check.restype = i64
        L.orc_lpa_async.argtypes = L.orc_lpa_sync.argtypes
        L.orc_lpa_async.restype = ct.c_int
        L.orc_lpa_async_waves.argtypes = [i64, P, P, P, dbl, ct.c_int, ct.c_int, ct.c_int, P, P, i32, P, P, P, P, P, P]
        L.orc_lpa_async_waves.restype = ct.c_int
        L.orc_sweep_range.argtypes = [i64, P, P, P, ct.c_int, i64, i64, P, P]
        L.orc_sweep_range.restype = i64
        L.orc_sweep_window.argtypes = [i64, i64, P, P, P, P, ct.c_int, P]
        L.orc_sweep_window.restype = i64
        L.orc_label_weights.argtypes = [i64, P, P, P, P, P, P, P]
        L.orc_label_weights.restype = i64
        L.orc_ht_capacity.argtypes = [i64]
        L.orc_ht_capacity.restype = u32
        L.orc_ht_probe_slot.argtypes = [u32, u32, i32, ct.c_int]
        L.orc_ht_probe_slot.restype = u32
        L.orc_ht_build.argtypes = [i64, P, P, u32, ct.c_int, P, P, P]
        L.orc_ht_build.restype = ct.c_int
        L.orc_modularity.argtypes = [i64, P, P, P, P]
        L.orc_modularity.restype = dbl
        L.orc_modularity_exact.argtypes = [i64, P, P, P, P, P, P, P, P]
        L.orc_modularity_exact.restype = ct.c_int
        L.orc_violations.argtypes = [i64, P, P, P, P]
        L.orc_violations.restype = i64
        _lib = L
    return _lib


def _np(x, dtype):
    """torch tensor / sequence / numpy -> contiguous numpy array of `dtype` (CPU)."""
    if x is None:
        return None
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


class Graph:
    """Host copy of a CSR graph in the oracle's layout (int64 offsets, int32 indices,
    float32 weights or None for unit weights)."""

    def __init__(self, offsets, indices, weights=None):
        self.off = _np(offsets, np.int64)
        self.idx = _np(indices, np.int32)
        self.w = _np(weights, np.float32)
        self.n = self.off.size - 1
        self.m = self.idx.size

    @classmethod
    def of(cls, g):
        """From any object with offsets / indices / weights attributes."""
        return cls(g.offsets, g.indices, g.weights)


@dataclass
class RunResult:
    labels: np.ndarray
    active: np.ndarray
    dN: list
    iterations: int
    converged: bool
    edges: list = None       # CSR entries of the vertices each sweep processed


def _run(fn, g: Graph, tol, max_iters, pl_period, labels=None, active=None, start_iter=0):
    n = g.n
    C = np.arange(n, dtype=np.int32) if labels is None else _np(labels, np.int32).copy()
    A = np.ones(n, dtype=np.uint8) if active is None else _np(active, np.uint8).copy()
    dN = np.zeros(max(max_iters, 1), dtype=np.int64)
    it = np.zeros(1, np.int32)
    cv = np.zeros(1, np.int32)
    E = np.zeros(max(max_iters, 1), dtype=np.int64)
    rc = fn(n, _p(g.off), _p(g.idx), _p(g.w), float(tol), int(max_iters), int(pl_period),
            int(start_iter), _p(C), _p(A), _p(dN), _p(it), _p(cv), _p(E))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    iters = int(it[0])
    return RunResult(C, A, [int(x) for x in dN[start_iter:iters]], iters, bool(cv[0]),
                     [int(x) for x in E[start_iter:iters]])


def lpa_sync(g: Graph, tol=0.05, max_iters=20, pl_period=4, labels=None, active=None, start_iter=0, cc_period=0):
    """Synchronous (double-buffered) LPA: Algorithm 1 applied to frozen labels; with
    cc_period > 0 the Cross-Check of Section 4.1 after every cc_period-th sweep."""
    if cc_period:
        L = lib()
        return _run(lambda n, o, i, w, t, m, p, s, *rest: L.orc_lpa_sync_cc(n, o, i, w, t, m, p, int(cc_period), s,
                                                                              *rest),
                    g, tol, max_iters, pl_period, labels, active, start_iter)
    return _run(lib().orc_lpa_sync, g, tol, max_iters, pl_period, labels, active, start_iter)


def cross_check(labels, prev):
    """The Cross-Check of one sweep (Section 4.1) on host arrays: returns (labels after the
    reverts, number reverted)."""
    C = _np(labels, np.int32).copy()
    P = _np(prev, np.int32)
    k = lib().orc_cross_check(C.size, _p(C), _p(P))
    return C, int(k)


def lpa_async(g: Graph, tol=0.05, max_iters=20, pl_period=4, labels=None, active=None, start_iter=0):
    """Asynchronous in-place LPA, vertices visited in order 0..n-1 (Section 4 item 1)."""
    return _run(lib().orc_lpa_async, g, tol, max_iters, pl_period, labels, active, start_iter)


def lpa_async_waves(g: Graph, wave_of, tol=0.05, max_iters=20, pl_period=4, labels=None, active=None,
                    start_iter=0, take_of=None):
    """Asynchronous LPA under a wave schedule: each sweep runs the waves 0, 1, ... in turn;
    vertex i takes its processed flag when wave take_of[i] starts (default: wave_of[i]) and
    decides in wave wave_of[i], on the labels as they stand when that wave starts; a wave's
    moves and marks land at its end.  One vertex per wave in id order is lpa_async; a single
    wave is lpa_sync."""
    W = _np(wave_of, np.int32)
    if W.size != g.n:
        raise ValueError("wave_of needs one entry per vertex")
    T = None if take_of is None else _np(take_of, np.int32)
    if T is not None and T.size != g.n:
        raise ValueError("take_of needs one entry per vertex")
    n_waves = int(W.max()) + 1 if W.size else 1
    L = lib()
    out = _run(lambda n, o, i, w, t, m, p, s, *rest: _waves_rc(L.orc_lpa_async_waves(n, o, i, w, t, m, p, s, _p(W),
                                                                                       _p(T), n_waves, *rest)),
               g, tol, max_iters, pl_period, labels, active, start_iter)
    return out


def _waves_rc(rc):
    if rc == -2:
        raise ValueError("wave index outside [0, n_waves), or a flag taken after its vertex decides")
    return rc


_mc = None


def _mc_lib():
    global _mc
    if _mc is None:
        build()
        L = ct.CDLL(_MC_LIB)
        P = ct.c_void_p
        L.mc_lpa_sync.argtypes = [ct.c_int64, P, P, P, ct.c_double, ct.c_int, ct.c_int, ct.c_int, P, P, P, P, P, P,
                                  ct.c_int]
        L.mc_lpa_sync.restype = ct.c_int
        L.mc_threads.restype = ct.c_int
        _mc = L
    return _mc


def multicore_threads() -> int:
    return int(_mc_lib().mc_threads())


def multicore_lpa_sync(g: Graph, tol=0.05, max_iters=20, pl_period=4, labels=None, active=None, start_iter=0,
                       threads=0):
    """The synchronous run of lpa_sync on all host cores (OpenMP); threads <= 0: all."""
    L = _mc_lib()
    return _run(lambda *a: L.mc_lpa_sync(*a, int(threads)), g, tol, max_iters, pl_period, labels, active,
                start_iter)


def sweep_range(g: Graph, labels, v0: int, v1: int, pl: bool = False):
    """New labels of vertices [v0, v1) after one all-active synchronous sweep on `labels`.
    Returns (labels_out, entries_scanned)."""
    C = _np(labels, np.int32)
    out = np.empty(v1 - v0, dtype=np.int32)
    e = lib().orc_sweep_range(g.n, _p(g.off), _p(g.idx), _p(g.w), int(pl), int(v0), int(v1), _p(C), _p(out))
    if e < 0:
        raise MemoryError("oracle allocation failed")
    return out, int(e)


def sweep_window(v0: int, v1: int, off_w, idx_w, w_w, labels, pl: bool = False):
    """sweep_range on a window of rows: off_w = offsets[v0:v1+1] (absolute), idx_w / w_w =
    the entries offsets[v0]:offsets[v1]; labels = all n labels.  Returns (new labels, entries)."""
    ow = _np(off_w, np.int64)
    iw = _np(idx_w, np.int32)
    ww = _np(w_w, np.float32)
    C = _np(labels, np.int32)
    out = np.empty(v1 - v0, dtype=np.int32)
    e = lib().orc_sweep_window(int(v0), int(v1), _p(ow), _p(iw), _p(ww), _p(C), int(pl), _p(out))
    if e < 0:
        raise MemoryError("oracle allocation failed")
    return out, int(e)


def label_weights(g: Graph, labels, i: int):
    """{label: float32 weight} of vertex i (sort-and-count)."""
    C = _np(labels, np.int32)
    d = int(g.off[i + 1] - g.off[i])
    lab = np.empty(max(d, 1), np.int32)
    s = np.empty(max(d, 1), np.float32)
    scratch = ct.create_string_buffer(max(d, 1) * 24)
    nd = lib().orc_label_weights(i, _p(g.off), _p(g.idx), _p(g.w), _p(C), _p(lab), _p(s),
                                 ct.cast(scratch, ct.c_void_p))
    return {int(lab[k]): float(s[k]) for k in range(nd)}


def ht_capacity(degree: int) -> int:
    return int(lib().orc_ht_capacity(int(degree)))


def ht_probe_slot(p1: int, k: int, t: int) -> int:
    return int(lib().orc_ht_probe_slot(p1, 2 * p1 + 1, k, t))


def ht_build(keys, vals, p1: int, max_retries: int = MAX_RETRIES):
    """Table (H_k, H_v) after inserting the pairs in order; returns (Hk, Hv, fallbacks)."""
    k = _np(keys, np.int32)
    v = _np(vals, np.float32)
    Hk = np.empty(p1, np.int32)
    Hv = np.empty(p1, np.float32)
    fb = np.zeros(1, np.int64)
    rc = lib().orc_ht_build(k.size, _p(k), _p(v), p1, max_retries, _p(Hk), _p(Hv), _p(fb))
    if rc != 0:
        raise RuntimeError("hashtable insert failed")
    return Hk, Hv, int(fb[0])


def modularity(g: Graph, labels) -> float:
    C = _np(labels, np.int32)
    return float(lib().orc_modularity(g.n, _p(g.off), _p(g.idx), _p(g.w), _p(C)))


def modularity_exact(g: Graph, labels) -> Fraction:
    """Exact Q as a Fraction (integer weights only)."""
    C = _np(labels, np.int32)
    nh, dh = np.zeros(1, np.int64), np.zeros(1, np.int64)
    nl, dl = np.zeros(1, np.uint64), np.zeros(1, np.uint64)
    rc = lib().orc_modularity_exact(g.n, _p(g.off), _p(g.idx), _p(g.w), _p(C), _p(nh), _p(nl), _p(dh), _p(dl))
    if rc != 0:
        raise ValueError("non-integer weights")
    num = (int(nh[0]) << 64) + int(nl[0])
    den = (int(dh[0]) << 64) + int(dl[0])
    return Fraction(0) if den == 0 else Fraction(num, den)


def violations(g: Graph, labels) -> int:
    C = _np(labels, np.int32)
    return int(lib().orc_violations(g.n, _p(g.off), _p(g.idx), _p(g.w), _p(C)))
