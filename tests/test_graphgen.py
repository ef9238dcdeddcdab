"""Input generators: counter-based hashing, CSR validity, symmetry, shapes; the GPU-marked
tests check that CPU and GPU generation agree."""
import pytest
import torch

from paper_2411_11468_gb300 import graphgen as gg


def test_splitmix64_known_output():
    """SplitMix64 seeded with state 0 produces 0xe220a8397b1dcdaf first
    (Steele, Lea, Flood 2014; the state is advanced by the golden gamma before mixing)."""
    assert gg.mix64_int(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF
    t = gg.mix64(torch.tensor([gg._s64(0x9E3779B97F4A7C15)], dtype=torch.int64))
    assert (int(t[0]) & gg.MASK64) == 0xE220A8397B1DCDAF


def test_tensor_hash_matches_python_ints():
    xs = [0, 1, 2, 12345, (1 << 63) - 1, 1 << 63, (1 << 64) - 1, 0xDEADBEEFCAFEBABE]
    t = gg.mix64(torch.tensor([gg._s64(x) for x in xs], dtype=torch.int64))
    assert [int(v) & gg.MASK64 for v in t] == [gg.mix64_int(x) for x in xs]


def _check_csr(g, self_loops_allowed=False):
    off, idx = g.offsets, g.indices.to(torch.int64)
    n = g.n
    assert off[0] == 0 and off[-1] == g.m
    assert bool((off[1:] >= off[:-1]).all())
    assert bool(((idx >= 0) & (idx < n)).all())
    u = torch.repeat_interleave(torch.arange(n), off[1:] - off[:-1])
    if not self_loops_allowed:
        assert bool((u != idx).all())
    keys = u * n + idx
    assert torch.unique(keys).numel() == keys.numel()          # no duplicates
    rev = torch.sort(idx * n + u).values
    assert torch.equal(rev, torch.sort(keys).values)            # symmetric
    if g.weights is not None:
        order_f = torch.argsort(keys)
        order_r = torch.argsort(idx * n + u)
        assert torch.equal(g.weights[order_f], g.weights[order_r])


def test_rmat_small_valid_and_deterministic():
    g = gg.rmat(12, weights="int8")
    _check_csr(g)
    assert g.weights.min() >= 1 and g.weights.max() <= 8
    assert torch.equal(g.weights, torch.round(g.weights))
    g2 = gg.rmat(12, weights="int8")
    assert torch.equal(g.offsets, g2.offsets) and torch.equal(g.indices, g2.indices)
    assert torch.equal(g.weights, g2.weights)
    deg = g.degrees()
    assert int(torch.argmax(deg)) == 0          # no permutation: vertex 0 is the top hub


def test_sbm_shape():
    g = gg.sbm(10_000, 100, 16.0, 2.0, seed=0)
    _check_csr(g)
    n = g.n
    u = torch.repeat_interleave(torch.arange(n), g.degrees())
    same = g.planted[u] == g.planted[g.indices.long()]
    d_in = same.sum().item() / n
    d_out = (~same).sum().item() / n
    assert abs(d_in - 16.0) < 0.3
    assert abs(d_out - 2.0) < 0.1


def test_batch_specs_ranges():
    specs = gg.batch_specs(256)
    assert all(100 <= s["n"] <= 100_000 for s in specs)
    assert all(2 <= s["block"] <= 1000 for s in specs)
    assert all(4 * 8 / 9 - 1e-9 <= s["d_in"] <= 32 * 8 / 9 + 1e-9 for s in specs)
    g = gg.batch_graph(specs[0])
    _check_csr(g)


def test_fixtures():
    g = gg.complete_bipartite(3)
    _check_csr(g)
    assert g.m == 18
    s = gg.star(4)
    assert s.degrees().tolist() == [4, 1, 1, 1, 1]


@pytest.mark.gpu
@pytest.mark.parametrize("scale,weights", [(12, "int8"), (14, "unit"), (16, "int8")])
def test_rmat_cpu_and_gpu_generation_agree(scale, weights):
    """The large R-MAT workloads are generated on the GPU; the CPU generator (which the oracle
    tests use) gives the same CSR at small scales."""
    a = gg.rmat(scale, weights=weights, device="cpu")
    b = gg.rmat(scale, weights=weights, device="cuda").to("cpu")
    assert torch.equal(a.offsets, b.offsets) and torch.equal(a.indices, b.indices)
    assert torch.equal(a.weights, b.weights)


@pytest.mark.gpu
def test_sbm_cpu_and_gpu_generation_agree():
    a = gg.sbm(10_000, 100, 16.0, 2.0, seed=0, device="cpu")
    b = gg.sbm(10_000, 100, 16.0, 2.0, seed=0, device="cuda").to("cpu")
    assert torch.equal(a.offsets, b.offsets) and torch.equal(a.indices, b.indices)
