"""lpa_modularity_noalloc, called through the C ABI, against the oracle's Eq. 1 and against
lpa_modularity on the same labels.

The no-allocation entry point serves callers that cannot allocate device memory; it keeps its
scratch in a fixed array compiled into the library, shared by every call.  Two calls in a row
must both agree with the handle-based modularity (the second call finds the first call's
contents in the shared array and must clear them).  This file is collected last.
"""
import ctypes as ct

import pytest
import torch

import oracle
from paper_2411_11468_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    from paper_2411_11468_gb300 import build
    build.build()
    from paper_2411_11468_gb300 import lpa
    L = lpa.load()
    P, i64 = ct.c_void_p, ct.c_int64
    L.lpa_modularity_noalloc.argtypes = [P, P, P, P, i64, i64, P, ct.POINTER(ct.c_double)]
    L.lpa_modularity_noalloc.restype = ct.c_int
    return lpa, L


def noalloc_q(L, csr, labels, stream):
    q = ct.c_double(float("nan"))
    w = None if csr.weights is None else ct.c_void_p(csr.weights.data_ptr())
    rc = L.lpa_modularity_noalloc(ct.c_void_p(csr.offsets.data_ptr()), ct.c_void_p(csr.indices.data_ptr()), w,
                                  ct.c_void_p(labels.data_ptr()), csr.n, csr.m, ct.c_void_p(stream.cuda_stream),
                                  ct.byref(q))
    return rc, q.value


@pytest.mark.parametrize("which", ["rmat-int", "sbm-unit", "rmat-dyadic"])
def test_noalloc_matches_handle_modularity_twice(libs, which):
    lpa, L = libs
    if which == "rmat-int":
        csr = gg.rmat(14, weights="int8")
    elif which == "sbm-unit":
        csr = gg.sbm(20_000, 100, 12.0, 3.0, seed=2, weights="none")
    else:
        base = gg.rmat(13, weights="unit")
        u = torch.repeat_interleave(torch.arange(base.n), base.degrees())
        key = torch.minimum(u, base.indices.long()) * base.n + torch.maximum(u, base.indices.long())
        w = torch.tensor([0.5, 1.25, 2.75])[gg.draws53(5, 9, key) % 3].to(torch.float32)
        csr = gg.CSRGraph(base.offsets, base.indices, w)
    dev = csr.to("cuda")
    stream = torch.cuda.current_stream()
    g = lpa.Graph(dev.offsets, dev.indices, dev.weights)
    g.run(0.05, 20, 4, lpa.SYNC)
    labels = g.labels()
    q_ref = g.modularity()
    q_orc = oracle.modularity(oracle.Graph.of(csr), labels.cpu())
    for _ in range(2):
        rc, q = noalloc_q(L, dev, labels, stream)
        assert rc == lpa.OK
        assert abs(q - q_orc) < 1e-12, (q, q_orc)
        assert abs(q - q_ref) < 1e-12, (q, q_ref)
    # a different labelling right after: the shared scratch must not leak the previous sums
    ident = torch.arange(dev.n, dtype=torch.int32, device="cuda")
    g.set_labels(ident)
    q_ref2 = g.modularity()
    rc, q2 = noalloc_q(L, dev, ident, stream)
    assert rc == lpa.OK and abs(q2 - q_ref2) < 1e-12
    assert abs(q2 - oracle.modularity(oracle.Graph.of(csr), ident.cpu())) < 1e-12


def test_noalloc_rejects_oversized_and_bad_labels(libs):
    lpa, L = libs
    csr = gg.rmat(10, weights="int8").to("cuda")
    labels = torch.zeros(csr.n, dtype=torch.int32, device="cuda")
    q = ct.c_double()
    rc = L.lpa_modularity_noalloc(ct.c_void_p(csr.offsets.data_ptr()), ct.c_void_p(csr.indices.data_ptr()),
                                  ct.c_void_p(csr.weights.data_ptr()), ct.c_void_p(labels.data_ptr()),
                                  (1 << 20) + 1, csr.m, None, ct.byref(q))
    assert rc == lpa.EINVAL
    assert b"scratch limit" in L.lpa_last_error()
    bad = torch.full((csr.n,), csr.n + 5, dtype=torch.int32, device="cuda")     # labels out of range
    rc, _ = noalloc_q(L, csr, bad, torch.cuda.current_stream())
    assert rc == lpa.EINVAL
    rc, q = noalloc_q(L, csr, labels, torch.cuda.current_stream())           # still usable afterwards
    assert rc == lpa.OK
