"""Python binding of liblpa.so (ctypes): argument marshalling only.

Every step of label propagation runs in the library's CUDA kernels; this module passes
pointers, sizes and the current torch CUDA stream.  It raises if liblpa.so is missing:
there is no CPU fallback.

    from paper_2411_11468_gb300 import lpa
    g = lpa.Graph(offsets, indices, weights)          # torch tensors (CPU or CUDA)
    st = g.run(tolerance=0.05, max_iters=20, pl_period=4, mode=lpa.SYNC)
    labels = g.labels()                                # torch.int32 on the graph's device
    q = g.modularity()
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblpa.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE, ECANCELED = 0, -1, -2, -3, -4, -5, -6
SYNC, ASYNC, RESUME = 0, 1, 16
OFFSETS_I32, OFFSETS_I64, HOST_PTRS, DEVICE_PTRS, CHECK_SYMMETRIC = 0, 1, 0, 2, 4
BORROW_INPUTS = 8
STATS_MAX_ITERS = 64
NUM_KERNELS = 12
KERNEL_NAMES = ["thread", "group", "warp", "cta", "cta_large", "cta_xl", "hub_begin", "hub_acc", "hub_clear",
                "hub_move", "hub_mark", "apply"]

SYMBOLS = ["lpa_create", "lpa_run", "lpa_labels", "lpa_modularity", "lpa_set_labels", "lpa_get_state",
           "lpa_set_state", "lpa_set_stream", "lpa_get_tuning", "lpa_set_tuning", "lpa_num_vertices",
           "lpa_num_entries", "lpa_device_bytes", "lpa_destroy", "lpa_strerror", "lpa_last_error",
           "lpa_kernel_name", "lpa_struct_size", "lpa_batch_create", "lpa_batch_run", "lpa_batch_labels",
           "lpa_batch_modularity", "lpa_batch_graph", "lpa_batch_size", "lpa_batch_device_bytes", "lpa_batch_destroy",
           "lpa_server_create", "lpa_server_submit", "lpa_server_step", "lpa_server_poll", "lpa_server_result",
           "lpa_server_clock", "lpa_server_device_bytes", "lpa_server_destroy", "lpa_batch_get_tuning",
           "lpa_batch_set_tuning", "lpa_autotune", "lpa_batch_autotune", "lpa_modularity_noalloc", "lpa_run_cc", "lpa_server_cancel", "lpa_trim_memory",
           "lpa_debug_fail_allocations"]


class LpaError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {_strerror(status)} ({status}){': ' + detail if detail else ''}")


class Stats(ct.Structure):
    _fields_ = [
        ("time_kernels", ct.c_int32),
        ("iterations", ct.c_int32),
        ("converged", ct.c_int32),
        ("first_iter", ct.c_int32),
        ("changed", ct.c_int64 * STATS_MAX_ITERS),
        ("active", ct.c_int64 * STATS_MAX_ITERS),
        ("edges", ct.c_int64 * STATS_MAX_ITERS),
        ("marks", ct.c_int64 * STATS_MAX_ITERS),
        ("iter_ms", ct.c_float * STATS_MAX_ITERS),
        ("total_ms", ct.c_float),
        ("launches", ct.c_int32),
        ("probe_fallbacks", ct.c_int64),
        ("kernel_ms", (ct.c_float * NUM_KERNELS) * STATS_MAX_ITERS),
        ("kernel_edges", (ct.c_int64 * NUM_KERNELS) * STATS_MAX_ITERS),
        ("kernel_active", (ct.c_int64 * NUM_KERNELS) * STATS_MAX_ITERS),
    ]

    @property
    def count(self) -> int:
        return min(self.iterations - self.first_iter, STATS_MAX_ITERS)

    def dN(self) -> list[int]:
        return [int(self.changed[i]) for i in range(self.count)]

    def to_dict(self) -> dict:
        k = self.count
        d = dict(iterations=self.iterations, converged=bool(self.converged), first_iter=self.first_iter,
                 changed=self.dN(), active=[int(self.active[i]) for i in range(k)],
                 edges=[int(self.edges[i]) for i in range(k)], marks=[int(self.marks[i]) for i in range(k)],
                 iter_ms=[float(self.iter_ms[i]) for i in range(k)], total_ms=float(self.total_ms),
                 probe_fallbacks=int(self.probe_fallbacks), launches=int(self.launches))
        if self.time_kernels:
            d["kernel_ms"] = [[float(self.kernel_ms[i][j]) for j in range(NUM_KERNELS)] for i in range(k)]
            d["kernel_edges"] = [[int(self.kernel_edges[i][j]) for j in range(NUM_KERNELS)] for i in range(k)]
            d["kernel_active"] = [[int(self.kernel_active[i][j]) for j in range(NUM_KERNELS)] for i in range(k)]
        return d


class Tuning(ct.Structure):
    _fields_ = [(name, ct.c_int32) for name in (
        "thread_max", "group_max", "group_lanes", "warp_max", "cta_max", "cta_threads", "cta_large_max",
        "cta_large_threads", "hub_chunk", "hub_table_shift", "smem_table_shift", "cta_xl_max",
        "cta_xl_threads", "item_vertices", "float_values", "hub_cluster", "probe", "flat_buckets", "hub_two_pass")] + \
        [("reserved", ct.c_int32 * 1)]

    def to_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}

    def update(self, **kw) -> "Tuning":
        """Sets the named fields (an unknown name raises KeyError instead of being ignored)."""
        names = {f for f, _ in self._fields_ if f != "reserved"}
        for k, v in kw.items():
            if k not in names:
                raise KeyError(f"lpa_tuning has no field {k!r}")
            setattr(self, k, int(v))
        return self


_lib = None


def load() -> ct.CDLL:
    """Loads liblpa.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"liblpa.so not built at {LIB_PATH}; run paper_2411_11468_gb300.build.build()")
    L = ct.CDLL(LIB_PATH)
    P, i64, i32 = ct.c_void_p, ct.c_int64, ct.c_int
    L.lpa_create.argtypes = [P, P, P, i64, i64, i32, P, ct.POINTER(P)]
    L.lpa_run.argtypes = [P, ct.c_double, i32, i32, i32, ct.POINTER(Stats)]
    L.lpa_run_cc.argtypes = [P, ct.c_double, i32, i32, i32, i32, ct.POINTER(Stats)]
    L.lpa_labels.argtypes = [P, P, i64, i32]
    L.lpa_modularity.argtypes = [P, ct.POINTER(ct.c_double)]
    L.lpa_set_labels.argtypes = [P, P, i64, i32]
    L.lpa_get_state.argtypes = [P, P, P, ct.POINTER(ct.c_int32), i64, i32]
    L.lpa_set_state.argtypes = [P, P, P, ct.c_int32, i64, i32]
    L.lpa_set_stream.argtypes = [P, P]
    L.lpa_get_tuning.argtypes = [P, ct.POINTER(Tuning)]
    L.lpa_set_tuning.argtypes = [P, ct.POINTER(Tuning)]
    for f in ("lpa_num_vertices", "lpa_num_entries", "lpa_device_bytes"):
        getattr(L, f).argtypes = [P]
        getattr(L, f).restype = i64
    L.lpa_destroy.argtypes = [P]
    L.lpa_destroy.restype = None
    L.lpa_strerror.argtypes = [i32]
    L.lpa_strerror.restype = ct.c_char_p
    L.lpa_last_error.argtypes = []
    L.lpa_last_error.restype = ct.c_char_p
    L.lpa_kernel_name.argtypes = [i32]
    L.lpa_kernel_name.restype = ct.c_char_p
    L.lpa_struct_size.argtypes = [i32]
    L.lpa_struct_size.restype = ct.c_size_t
    if L.lpa_struct_size(0) != ct.sizeof(Stats) or L.lpa_struct_size(1) != ct.sizeof(Tuning):
        raise RuntimeError("liblpa.so struct layout does not match the binding")
    _lib = L
    return L


def _strerror(status: int) -> str:
    try:
        return load().lpa_strerror(status).decode()
    except Exception:
        return "error"


def _check(status: int, where: str):
    if status != OK:
        detail = load().lpa_last_error().decode(errors="replace")
        raise LpaError(status, where, detail)


def _ptr(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _stream_handle(device) -> ct.c_void_p:
    if device.type != "cuda":
        return ct.c_void_p(None)
    return ct.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Graph:
    """A CSR graph resident on the current CUDA device (owned by liblpa.so).

    offsets: int32 or int64 [n+1]; indices: int32 [m]; weights: float32 [m] or None (unit).
    Tensors may live on the host (copied to the device) or on the current CUDA device.
    The handle uses torch's current CUDA stream at creation (or `stream`).
    """

    def __init__(self, offsets, indices, weights=None, check_symmetric: bool = False, stream=None):
        L = load()
        if not torch.cuda.is_available():
            raise RuntimeError("liblpa needs a CUDA device")
        offsets = offsets.contiguous()
        indices = indices.contiguous()
        if indices.dtype != torch.int32:
            raise TypeError("indices must be int32")
        if offsets.dtype not in (torch.int32, torch.int64):
            raise TypeError("offsets must be int32 or int64")
        if weights is not None:
            weights = weights.contiguous()
            if weights.dtype != torch.float32:
                raise TypeError("weights must be float32")
        on_dev = offsets.is_cuda
        for t in (indices, weights):
            if t is not None and t.is_cuda != on_dev:
                raise ValueError("offsets, indices and weights must be on the same device")
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.n = offsets.numel() - 1
        self.m = indices.numel()
        flags = (OFFSETS_I64 if offsets.dtype == torch.int64 else OFFSETS_I32)
        flags |= DEVICE_PTRS if on_dev else HOST_PTRS
        if check_symmetric:
            flags |= CHECK_SYMMETRIC
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = ct.c_void_p()
        _check(L.lpa_create(_ptr(offsets), _ptr(indices), _ptr(weights), self.n, self.m, flags,
                            ct.c_void_p(stream.cuda_stream), ct.byref(h)), "lpa_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().lpa_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- algorithm ------------------------------------------------------------------
    def run(self, tolerance: float = 0.05, max_iters: int = 20, pl_period: int = 4, mode: int = SYNC,
            resume: bool = False, time_kernels: bool = False, cc_period: int = 0) -> Stats:
        """lpa_run, or lpa_run_cc when cc_period > 0 (Cross-Check every cc_period sweeps)."""
        st = Stats()
        st.time_kernels = 1 if time_kernels else 0
        m = int(mode) | (RESUME if resume else 0)
        if cc_period:
            _check(load().lpa_run_cc(self._h, float(tolerance), int(max_iters), int(pl_period), int(cc_period), m,
                                     ct.byref(st)), "lpa_run_cc")
        else:
            _check(load().lpa_run(self._h, float(tolerance), int(max_iters), int(pl_period), m, ct.byref(st)),
                   "lpa_run")
        return st

    def labels(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.n, dtype=torch.int32, device=self.device)
        if out.dtype != torch.int32 or out.numel() != self.n or not out.is_contiguous():
            raise ValueError("out must be a contiguous int32 tensor of n elements")
        _check(load().lpa_labels(self._h, _ptr(out), self.n, 1 if out.is_cuda else 0), "lpa_labels")
        return out

    def modularity(self) -> float:
        q = ct.c_double()
        _check(load().lpa_modularity(self._h, ct.byref(q)), "lpa_modularity")
        return q.value

    def set_labels(self, labels: torch.Tensor):
        labels = labels.to(torch.int32).contiguous()
        _check(load().lpa_set_labels(self._h, _ptr(labels), labels.numel(), 1 if labels.is_cuda else 0),
               "lpa_set_labels")

    def get_state(self):
        C = torch.empty(self.n, dtype=torch.int32)
        A = torch.empty(self.n, dtype=torch.uint8)
        it = ct.c_int32()
        _check(load().lpa_get_state(self._h, _ptr(C), _ptr(A), ct.byref(it), self.n, 0), "lpa_get_state")
        return C, A, it.value

    def set_state(self, labels, unprocessed, next_iter: int):
        labels = None if labels is None else labels.to(torch.int32).contiguous()
        unprocessed = None if unprocessed is None else unprocessed.to(torch.uint8).contiguous()
        dev = [t.is_cuda for t in (labels, unprocessed) if t is not None]
        on_dev = 1 if (dev and dev[0]) else 0
        _check(load().lpa_set_state(self._h, _ptr(labels), _ptr(unprocessed), int(next_iter), self.n, on_dev),
               "lpa_set_state")

    def tuning(self) -> Tuning:
        t = Tuning()
        _check(load().lpa_get_tuning(self._h, ct.byref(t)), "lpa_get_tuning")
        return t

    def set_tuning(self, t: Tuning | None = None, **kw):
        if t is None:
            t = self.tuning()
        t.update(**kw)
        _check(load().lpa_set_tuning(self._h, ct.byref(t)), "lpa_set_tuning")

    def autotune(self, tolerance=0.05, max_iters=20, pl_period=4, mode=SYNC, reps=2):
        """lpa_autotune: returns (tuning dict, best ms, configurations timed); the best tuning
        stays installed."""
        t, ms, k = Tuning(), ct.c_float(), ct.c_int()
        _check(_load_multi().lpa_autotune(self._h, float(tolerance), int(max_iters), int(pl_period), int(mode),
                                          int(reps), ct.byref(t), ct.byref(ms), ct.byref(k)), "lpa_autotune")
        return t.to_dict(), ms.value, k.value

    def set_stream(self, stream):
        self.stream = stream
        _check(load().lpa_set_stream(self._h, ct.c_void_p(stream.cuda_stream)), "lpa_set_stream")

    def device_bytes(self) -> int:
        return int(load().lpa_device_bytes(self._h))


# ----------------------------------------------------------------------------------------
# batches and the request server

class GraphDesc(ct.Structure):
    _fields_ = [("offsets", ct.c_void_p), ("indices", ct.c_void_p), ("weights", ct.c_void_p),
                ("n_vertices", ct.c_int64), ("n_entries", ct.c_int64)]


class Result(ct.Structure):
    _fields_ = [("iterations", ct.c_int32), ("converged", ct.c_int32), ("last_changed", ct.c_int64)]

    def to_dict(self):
        return dict(iterations=self.iterations, converged=bool(self.converged), last_changed=self.last_changed)


_multi_ready = False


def debug_fail_allocations(after: int):
    """lpa_debug_fail_allocations: device allocations fail after `after` more (< 0: off)."""
    L = load()
    L.lpa_debug_fail_allocations.argtypes = [ct.c_longlong]
    L.lpa_debug_fail_allocations.restype = None
    L.lpa_debug_fail_allocations(int(after))


def trim_memory():
    """lpa_trim_memory: returns the device memory cached by destroyed handles to the driver."""
    L = load()
    L.lpa_trim_memory.argtypes = []
    L.lpa_trim_memory.restype = ct.c_int
    _check(L.lpa_trim_memory(), "lpa_trim_memory")


def _load_multi():
    global _multi_ready
    L = load()
    if _multi_ready:
        return L
    P, i32, i64 = ct.c_void_p, ct.c_int, ct.c_int64
    L.lpa_batch_create.argtypes = [i32, ct.POINTER(GraphDesc), i32, P, ct.POINTER(P)]
    L.lpa_batch_run.argtypes = [P, ct.c_double, i32, i32, i32, ct.POINTER(Result), ct.POINTER(ct.c_float)]
    L.lpa_batch_labels.argtypes = [P, i32, P, i64, i32]
    L.lpa_batch_modularity.argtypes = [P, ct.POINTER(ct.c_double)]
    L.lpa_batch_graph.argtypes = [P, i32, ct.POINTER(P)]
    L.lpa_batch_get_tuning.argtypes = [P, ct.POINTER(Tuning)]
    L.lpa_batch_set_tuning.argtypes = [P, ct.POINTER(Tuning)]
    L.lpa_autotune.argtypes = [P, ct.c_double, i32, i32, i32, i32, ct.POINTER(Tuning), ct.POINTER(ct.c_float),
                               ct.POINTER(ct.c_int)]
    L.lpa_batch_autotune.argtypes = [P, ct.c_double, i32, i32, i32, i32, ct.POINTER(Tuning),
                                     ct.POINTER(ct.c_float), ct.POINTER(ct.c_int)]
    L.lpa_batch_size.argtypes = [P]
    L.lpa_batch_device_bytes.argtypes = [P]
    L.lpa_batch_device_bytes.restype = i64
    L.lpa_batch_destroy.argtypes = [P]
    L.lpa_batch_destroy.restype = None
    L.lpa_server_create.argtypes = [ct.c_size_t, i32, P, ct.POINTER(P)]
    L.lpa_server_submit.argtypes = [P, ct.POINTER(GraphDesc), i32, ct.c_double, i32, i32, i32, ct.POINTER(ct.c_int64)]
    L.lpa_server_step.argtypes = [P, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]
    L.lpa_server_poll.argtypes = [P, ct.POINTER(ct.c_int64), i32, ct.POINTER(ct.c_int)]
    L.lpa_server_cancel.argtypes = [P, i64]
    L.lpa_server_result.argtypes = [P, i64, P, i64, ct.POINTER(Result), ct.POINTER(ct.c_double),
                                    ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
    L.lpa_server_clock.argtypes = [P]
    L.lpa_server_clock.restype = ct.c_double
    L.lpa_server_device_bytes.argtypes = [P]
    L.lpa_server_device_bytes.restype = i64
    L.lpa_server_destroy.argtypes = [P]
    L.lpa_server_destroy.restype = None
    _multi_ready = True
    return L


def _desc(offsets, indices, weights):
    return GraphDesc(offsets.data_ptr(), indices.data_ptr(), None if weights is None else weights.data_ptr(),
                     offsets.numel() - 1, indices.numel())


class _Borrowed(Graph):
    """A graph handle owned by a batch (not destroyed by this object)."""

    def __init__(self, handle, n, m, device):
        self._h = handle
        self.n, self.m, self.device = n, m, device

    def close(self):
        self._h = ct.c_void_p()


class Batch:
    """Many independent CSR graphs on the device, solved together (lpa_batch_*).

    graphs: list of (offsets, indices, weights) tensors, all on the host or all on the device,
    all offsets of one dtype (int32 or int64)."""

    def __init__(self, graphs, stream=None):
        L = _load_multi()
        self._keep = [tuple(t.contiguous() if t is not None else None for t in g) for g in graphs]
        if not self._keep:
            raise ValueError("empty batch")
        o0 = self._keep[0][0]
        flags = (OFFSETS_I64 if o0.dtype == torch.int64 else OFFSETS_I32) | (DEVICE_PTRS if o0.is_cuda else HOST_PTRS)
        descs = (GraphDesc * len(self._keep))(*[_desc(*g) for g in self._keep])
        self.sizes = [(g[0].numel() - 1, g[1].numel()) for g in self._keep]
        self.device = torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        h = ct.c_void_p()
        _check(L.lpa_batch_create(len(self._keep), descs, flags, ct.c_void_p(stream.cuda_stream), ct.byref(h)),
               "lpa_batch_create")
        self._h = h
        if not o0.is_cuda:
            self._keep = None

    def __len__(self):
        return len(self.sizes)

    def run(self, tolerance=0.05, max_iters=20, pl_period=4, mode=SYNC):
        res = (Result * len(self))()
        ms = ct.c_float()
        _check(_load_multi().lpa_batch_run(self._h, float(tolerance), int(max_iters), int(pl_period), int(mode),
                                           res, ct.byref(ms)), "lpa_batch_run")
        return [r.to_dict() for r in res], ms.value

    def labels(self, i, out=None):
        n = self.sizes[i][0]
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=self.device)
        _check(_load_multi().lpa_batch_labels(self._h, i, _ptr(out), n, 1 if out.is_cuda else 0), "lpa_batch_labels")
        return out

    def modularity(self):
        q = (ct.c_double * len(self))()
        _check(_load_multi().lpa_batch_modularity(self._h, q), "lpa_batch_modularity")
        return list(q)

    def graph(self, i) -> Graph:
        """Borrowed handle of graph i (lpa_run solves it alone on the same device data)."""
        h = ct.c_void_p()
        _check(_load_multi().lpa_batch_graph(self._h, i, ct.byref(h)), "lpa_batch_graph")
        return _Borrowed(h, self.sizes[i][0], self.sizes[i][1], self.device)

    def device_bytes(self):
        return int(_load_multi().lpa_batch_device_bytes(self._h))

    def tuning(self) -> Tuning:
        t = Tuning()
        _check(_load_multi().lpa_batch_get_tuning(self._h, ct.byref(t)), "lpa_batch_get_tuning")
        return t

    def set_tuning(self, t: Tuning | None = None, **kw):
        if t is None:
            t = self.tuning()
        t.update(**kw)
        _check(_load_multi().lpa_batch_set_tuning(self._h, ct.byref(t)), "lpa_batch_set_tuning")

    def autotune(self, tolerance=0.05, max_iters=20, pl_period=4, mode=SYNC, reps=2):
        """lpa_batch_autotune: returns (tuning dict, best device ms, configurations timed)."""
        t, ms, k = Tuning(), ct.c_float(), ct.c_int()
        _check(_load_multi().lpa_batch_autotune(self._h, float(tolerance), int(max_iters), int(pl_period), int(mode),
                                                int(reps), ct.byref(t), ct.byref(ms), ct.byref(k)),
               "lpa_batch_autotune")
        return t.to_dict(), ms.value, k.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _load_multi().lpa_batch_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (lpa_server_*): submit host CSR graphs, call step()
    repeatedly, collect finished requests."""

    def __init__(self, hbm_budget_bytes, max_resident=256):
        L = _load_multi()
        h = ct.c_void_p()
        _check(L.lpa_server_create(int(hbm_budget_bytes), int(max_resident), None, ct.byref(h)), "lpa_server_create")
        self._h = h
        self._sizes = {}
        self._borrowed = {}

    def submit(self, offsets, indices, weights=None, tolerance=0.05, max_iters=20, pl_period=4, mode=SYNC,
               borrow=False) -> int:
        """Queues a request.  borrow=True passes LPA_BORROW_INPUTS: the server reads the host
        tensors at admission (keep them unchanged; this object holds a reference until the
        result is collected)."""
        offsets = offsets.contiguous().cpu()
        indices = indices.contiguous().cpu()
        weights = None if weights is None else weights.contiguous().cpu()
        flags = (OFFSETS_I64 if offsets.dtype == torch.int64 else OFFSETS_I32) | (BORROW_INPUTS if borrow else 0)
        d = _desc(offsets, indices, weights)
        rid = ct.c_int64()
        _check(_load_multi().lpa_server_submit(self._h, ct.byref(d), flags, float(tolerance), int(max_iters),
                                               int(pl_period), int(mode), ct.byref(rid)), "lpa_server_submit")
        self._sizes[rid.value] = offsets.numel() - 1
        if borrow:
            self._borrowed[rid.value] = (offsets, indices, weights)
        return rid.value

    def step(self):
        c, r, q = ct.c_int(), ct.c_int(), ct.c_int()
        _check(_load_multi().lpa_server_step(self._h, ct.byref(c), ct.byref(r), ct.byref(q)), "lpa_server_step")
        return c.value, r.value, q.value

    def cancel(self, rid):
        _check(_load_multi().lpa_server_cancel(self._h, int(rid)), "lpa_server_cancel")

    def poll(self, max_ids=4096):
        ids = (ct.c_int64 * max_ids)()
        n = ct.c_int()
        _check(_load_multi().lpa_server_poll(self._h, ids, max_ids, ct.byref(n)), "lpa_server_poll")
        return [ids[i] for i in range(n.value)]

    def result(self, rid):
        n = self._sizes.pop(rid)
        self._borrowed.pop(rid, None)
        lab = torch.empty(n, dtype=torch.int32)
        res = Result()
        ts, ta, tf = ct.c_double(), ct.c_double(), ct.c_double()
        _check(_load_multi().lpa_server_result(self._h, rid, _ptr(lab), n, ct.byref(res), ct.byref(ts), ct.byref(ta),
                                               ct.byref(tf)), "lpa_server_result")
        self._borrowed.pop(rid, None)
        return lab, res.to_dict(), (ts.value, ta.value, tf.value)

    def clock(self):
        return float(_load_multi().lpa_server_clock(self._h))

    def device_bytes(self):
        return int(_load_multi().lpa_server_device_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _load_multi().lpa_server_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
