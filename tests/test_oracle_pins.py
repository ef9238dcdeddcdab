"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each case states its derivation.  Notation: Algorithm 1 (lpa, lpaMove), Algorithm 2
(hashtableAccumulate), Eq. 1 (modularity), Eq. 3 (update rule), Section 4 items
(1)-(5) (asynchronous update, 20 iterations, tolerance, pruning, strict tie-break).
"""
import os
import random
from collections import defaultdict
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2411_11468_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_form_traces.txt")


def G(csr):
    return oracle.Graph.of(csr)


# --------------------------------------------------------------------------------------
# closed-form traces (tests/golden/closed_form_traces.txt)

def _load_traces():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            case, mode, params, tol, mi, pl, dn, rule = [x.strip() for x in line.split("|")]
            p = dict(kv.split("=") for kv in params.split(","))
            p = {k: int(v) for k, v in p.items()}
            if "x" in dn:
                val, rep = dn.split("x")
                dns = [int(val)] * int(rep)
            else:
                dns = [int(x) for x in dn.split(",")]
            rows.append((case, mode, p, float(tol), int(mi), int(pl), dns, rule))
    return rows


def _graph_for(case, p):
    if case.startswith("cliques"):
        return gg.cliques(p["k"], p["s"])
    if case.startswith("bridge"):
        return gg.two_cliques_bridge(p["s"])
    if case.startswith("knn"):
        return gg.complete_bipartite(p["n"])
    if case.startswith("star"):
        return gg.star(p["n"])
    raise KeyError(case)


def _expected_labels(case, p, rule, n):
    if rule == "clique-min":
        return [(v // p["s"]) * p["s"] for v in range(n)]
    if rule == "A=0,B=s":
        s = p["s"]
        return [0] * s + [s] * s
    if rule == "all=0":
        return [0] * n
    return None


@pytest.mark.parametrize("row", _load_traces(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_closed_form_trace(row):
    """Derivations (unit weights, ties -> smallest label):

    cliques (k disjoint K_s, ids contiguous): l=0 is a PL iteration; every vertex but
      the clique minimum c0 sees s-1 labels of weight 1 and takes c0 (< own id); c0's
      best is c0+1 > c0, so PL blocks it.  dN = k(s-1).  l=1: all neighbours hold c0,
      nobody moves, dN/N = 0 < tau -> stop after 2 iterations.  Async (order 0..n-1)
      reaches the same labels: vertex c0+t sees c0 with weight t >= 1.
    bridge (K_s on [0,s), K_s on [s,2s), edge (s-1,s)), sync: l=0 (PL): A\\{0} -> 0,
      vertex s sees {s-1, s+1..2s-1} tied -> s-1 (< s), B\\{s} -> s; dN = 2s-1.
      l=1: vertex s sees label s with weight s-1 > 1 -> back to s; nobody else moves
      (for s >= 4 a vertex of B sees s with weight s-2 > 1); dN = 1.  If 1/(2s) < tau
      (s=12) the run stops here, else l=2 has dN = 0.
    bridge, async: l=0: vertex s already sees s-1 relabelled 0 and ties to 0; B then
      cascades to 0 (vertex s+t sees 0 with weight t+1); dN = (s-1) + 1 + (s-1)
      = 2s-1; l=1 dN = 0.
    K_{n,n}, no PL: A takes n, B takes 0, then they swap forever: dN = 2n each
      iteration up to the cap (the community swap of Section 4.1).
    K_{n,n}, PL every 4: l=0 blocks A (best n > a) and moves B to 0; l=1 moves A\\{0}
      to 0 (n-1 moves; B sees min label 0 = own); l=2 dN = 0.
    star K_{1,n}: l=0 blocks the centre, leaves move to 0; l=1 only the centre is
      active and keeps 0.
    """
    case, mode, p, tol, mi, pl, dns, rule = row
    g = G(_graph_for(case, p))
    run = oracle.lpa_sync if mode == "sync" else oracle.lpa_async
    r = run(g, tol, mi, pl)
    assert r.dN == dns
    assert r.iterations == len(dns)
    assert r.converged == (len(dns) < mi)
    exp = _expected_labels(case, p, rule, g.n)
    if exp is not None:
        assert r.labels.tolist() == exp
    if rule == "oscillating":
        n = p["n"]
        # after an even number of sweeps the labels are back to the first-sweep state of
        # the previous pair: A holds 0 and B holds n after 20 (even) sweeps
        assert r.labels.tolist() == [0] * n + [n] * n


def test_cliques_modularity_closed_form():
    """k equal cliques as communities: sigma_c = Sigma_c = s(s-1), 2m = k s(s-1), so
    Q = k (1/k - 1/k^2) = 1 - 1/k (Eq. 1)."""
    k, s = 5, 6
    g = G(gg.cliques(k, s))
    r = oracle.lpa_sync(g)
    assert oracle.modularity_exact(g, r.labels) == 1 - Fraction(1, k)
    assert abs(oracle.modularity(g, r.labels) - (1 - 1 / k)) < 1e-15


def test_bridge_modularity_closed_form():
    """Two K_s plus a bridge split into the two cliques: sigma = s(s-1) per side,
    Sigma = s(s-1)+1, 2m = 2s(s-1)+2: Q = 2[s(s-1)/(2m) - 1/4]."""
    s = 6
    g = G(gg.two_cliques_bridge(s))
    r = oracle.lpa_sync(g)
    two_m = 2 * s * (s - 1) + 2
    assert oracle.modularity_exact(g, r.labels) == 2 * (Fraction(s * (s - 1), two_m) - Fraction(1, 4))
    # the asynchronous run merges everything: single community, Q = 0
    ra = oracle.lpa_async(g)
    assert oracle.modularity_exact(g, ra.labels) == 0


# --------------------------------------------------------------------------------------
# hashtable (Section 4.2, Algorithm 2)

def test_capacity_reading():
    """p1 = nextPow2(D) - 1 with nextPow2 = smallest power of two strictly above D:
    the smallest 2^k - 1 that is >= D."""
    for d in range(1, 5000):
        p1 = oracle.ht_capacity(d)
        assert p1 == (1 << d.bit_length()) - 1
        assert p1 >= d and (p1 + 1) & p1 == 0
        assert p1 <= 2 * d - 1          # fits the 2*D_i reservation of Section 4.2


def test_probe_sequence_matches_unreduced_recurrence():
    """The oracle keeps i and delta reduced mod p1; Algorithm 2 lets them grow
    (i <- i + delta, delta <- 2 delta + (k mod p2)).  Slots s_t = i_t mod p1 agree."""
    rnd = random.Random(1)
    for p1 in [1, 3, 7, 15, 31, 255, 4095, (1 << 20) - 1]:
        p2 = 2 * p1 + 1
        for _ in range(20):
            k = rnd.randrange(0, 1 << 31)
            i, d = k, 1
            for t in range(40):
                assert oracle.ht_probe_slot(p1, k, t) == i % p1
                i = i + d
                d = 2 * d + (k % p2)


@pytest.mark.parametrize("k", range(1, 12))
def test_hashtable_equals_sort_and_count(k):
    """Per-vertex (key, sum) sets of the Algorithm 2 table equal a plain count, at
    D = 2^k - 1, 2^k, 2^k + 1, for few and for all-distinct keys; the failed path is
    never taken."""
    rnd = random.Random(k)
    for D in (2 ** k - 1, 2 ** k, 2 ** k + 1):
        for universe in (3, max(1, D // 4), 1 << 30):
            keys = [rnd.randrange(universe) for _ in range(D)]
            vals = [float(rnd.randint(1, 8)) for _ in range(D)]
            p1 = oracle.ht_capacity(D)
            Hk, Hv, fb = oracle.ht_build(keys, vals, p1)
            ref = defaultdict(float)
            for kk, vv in zip(keys, vals):
                ref[kk] += vv
            got = {int(a): float(b) for a, b in zip(Hk, Hv) if a != -1}
            assert got == dict(ref)
            assert len([a for a in Hk if a != -1]) == len(ref)   # each key in one slot
            assert fb <= D


def _alg2_unreduced(keys, vals, p1, max_retries=oracle.MAX_RETRIES):
    """Algorithm 2, single-threaded, with Python's unbounded integers: i <- k, delta <- 1;
    s = i mod p1; take s if empty or holding k; else i <- i + delta,
    delta <- 2 delta + (k mod p2).  After max_retries probes: linear scan from s."""
    p2 = 2 * p1 + 1
    Hk = [-1] * p1
    Hv = [0.0] * p1
    for k, v in zip(keys, vals):
        i, d = k, 1
        s = None
        for _ in range(max_retries):
            s = i % p1
            if Hk[s] in (k, -1):
                break
            i, d = i + d, 2 * d + (k % p2)
        else:
            for u in range(1, p1 + 1):
                q = (s + u) % p1
                if Hk[q] in (k, -1):
                    s = q
                    break
        Hk[s] = k
        Hv[s] += v
    return Hk, Hv


@pytest.mark.parametrize("seed", range(8))
def test_hashtable_layout_matches_unreduced_algorithm2(seed):
    """Same insertion order -> the same slot for every key (pins the probe recurrence
    and the fallback of the oracle's table, not only its contents)."""
    rnd = random.Random(300 + seed)
    for D in (1, 2, 3, 7, 8, 31, 32, 33, 255, 1000):
        keys = [rnd.randrange(1 << 31) if seed % 2 else rnd.randrange(max(1, D)) for _ in range(D)]
        vals = [float(rnd.randint(1, 8)) for _ in range(D)]
        p1 = oracle.ht_capacity(D)
        Hk, Hv, _ = oracle.ht_build(keys, vals, p1)
        rk, rv = _alg2_unreduced(keys, vals, p1)
        assert Hk.tolist() == rk
        assert Hv.tolist() == rv


def test_hashtable_full_table_uses_fallback():
    """A table filled to capacity (D = p1 distinct keys) still accepts every key: the
    linear fallback after MAX_RETRIES probes finds the remaining empty slots."""
    p1 = 15
    keys = list(range(0, 15 * 17, 17))          # 15 distinct keys, all = 2 (mod 15)
    Hk, Hv, fb = oracle.ht_build(keys, [1.0] * 15, p1)
    assert sorted(int(a) for a in Hk) == sorted(keys)
    assert fb >= 0


# --------------------------------------------------------------------------------------
# modularity (Eq. 1)

def _dense(g):
    n = g.n
    W = np.zeros((n, n))
    for i in range(n):
        for e in range(g.off[i], g.off[i + 1]):
            W[i, g.idx[e]] += 1.0 if g.w is None else g.w[e]
    return W


def _newman_pairwise(W, C):
    """(1/2m) sum_{i,j} [A_ij - K_i K_j / 2m] delta(C_i, C_j) over all ordered pairs."""
    K = W.sum(1)
    two_m = W.sum()
    q = Fraction(0)
    for i in range(len(C)):
        for j in range(len(C)):
            if C[i] == C[j]:
                q += Fraction(int(W[i, j])) - Fraction(int(K[i]) * int(K[j]), int(two_m))
    return q / int(two_m)


@pytest.mark.parametrize("seed", range(12))
def test_modularity_pairwise_bruteforce(seed):
    """Community form of Eq. 1 (oracle) = Newman's pairwise sum, exactly, N <= 10."""
    rnd = random.Random(seed)
    n = rnd.randint(2, 10)
    g = G(gg.random_small(n, 0.5, seed, self_loops=(seed % 3 == 0)))
    if g.m == 0:
        return
    W = _dense(g)
    for _ in range(5):
        C = [rnd.randrange(n) for _ in range(n)]
        q = _newman_pairwise(W, C)
        assert oracle.modularity_exact(g, C) == q
        assert abs(oracle.modularity(g, C) - float(q)) < 1e-14
        assert -0.5 <= float(q) <= 1.0


def test_modularity_special_partitions():
    """Single community: Q = 0.  Singletons (no self-loops): Q = -sum_i (K_i/2m)^2."""
    g = G(gg.random_small(40, 0.2, 7))
    K = _dense(g).sum(1)
    two_m = K.sum()
    assert oracle.modularity_exact(g, [0] * g.n) == 0
    sing = oracle.modularity_exact(g, list(range(g.n)))
    assert sing == -sum(Fraction(int(k), int(two_m)) ** 2 for k in K)


# --------------------------------------------------------------------------------------
# dense-matrix restatement of the synchronous and asynchronous sweeps (N <= 64)

def _best_dense(W, C, i):
    """Eq. 3 on a dense weight matrix: argmax over labels of non-self neighbours."""
    cand = {}
    for j in np.nonzero(W[i])[0]:
        if j == i:
            continue
        cand[C[j]] = cand.get(C[j], 0.0) + W[i, j]
    if not cand:
        return None
    mx = max(cand.values())
    return min(c for c, v in cand.items() if v == mx)


def _dense_sync(W, tol, max_iters, pl_period):
    n = W.shape[0]
    C = list(range(n))
    act = [True] * n
    dns, labels_per_iter = [], []
    for l in range(max_iters):
        pl = pl_period > 0 and l % pl_period == 0
        Cn = list(C)
        an = [False] * n
        ch = 0
        for i in range(n):
            if not act[i]:
                continue
            c = _best_dense(W, C, i)
            if c is not None and c != C[i] and (not pl or c < C[i]):
                Cn[i] = c
                ch += 1
                for j in np.nonzero(W[i])[0]:
                    an[j] = True
        C, act = Cn, an
        dns.append(ch)
        labels_per_iter.append(list(C))
        if not pl and ch / n < tol:
            break
    return dns, labels_per_iter


def _dense_async(W, tol, max_iters, pl_period):
    n = W.shape[0]
    C = list(range(n))
    act = [True] * n
    dns = []
    for l in range(max_iters):
        pl = pl_period > 0 and l % pl_period == 0
        ch = 0
        for i in range(n):
            if not act[i]:
                continue
            act[i] = False
            c = _best_dense(W, C, i)
            if c is not None and c != C[i] and (not pl or c < C[i]):
                C[i] = c
                ch += 1
                for j in np.nonzero(W[i])[0]:
                    act[j] = True
        dns.append(ch)
        if not pl and ch / n < tol:
            break
    return dns, C


@pytest.mark.parametrize("seed", range(16))
def test_sync_matches_dense_restatement_every_iteration(seed):
    rnd = random.Random(100 + seed)
    n = rnd.randint(5, 64)
    p = rnd.choice([0.05, 0.1, 0.2, 0.4])
    g = G(gg.random_small(n, p, seed, wmax=rnd.choice([1, 3, 8]), self_loops=(seed % 4 == 0)))
    W = _dense(g)
    tol, mi, pl = rnd.choice([0.0, 0.05, 0.2]), rnd.choice([5, 20]), rnd.choice([0, 2, 4])
    dns, per_iter = _dense_sync(W, tol, mi, pl)
    r = oracle.lpa_sync(g, tol, mi, pl)
    assert r.dN == dns
    assert r.labels.tolist() == per_iter[-1]
    for t in range(1, len(per_iter) + 1):       # labels after every iteration
        rt = oracle.lpa_sync(g, tol, t, pl)
        assert rt.labels.tolist() == per_iter[t - 1]


@pytest.mark.parametrize("seed", range(12))
def test_async_matches_dense_restatement(seed):
    rnd = random.Random(200 + seed)
    n = rnd.randint(5, 64)
    g = G(gg.random_small(n, rnd.choice([0.05, 0.15, 0.3]), 50 + seed, wmax=rnd.choice([1, 8])))
    W = _dense(g)
    dns, C = _dense_async(W, 0.05, 20, 4)
    r = oracle.lpa_async(g, 0.05, 20, 4)
    assert r.dN == dns
    assert r.labels.tolist() == C


def test_resume_equals_single_run():
    """State after k iterations (labels, active set, next iteration) resumes to the same
    result as an uninterrupted run (the whole state of Algorithm 1's loop)."""
    g = G(gg.sbm(600, 30, 8, 2, seed=3, weights="int8"))
    full = oracle.lpa_sync(g, 0.0, 12, 4)
    part = oracle.lpa_sync(g, 0.0, 5, 4)
    rest = oracle.lpa_sync(g, 0.0, 12, 4, labels=part.labels, active=part.active, start_iter=part.iterations)
    assert rest.labels.tolist() == full.labels.tolist()
    assert part.dN + rest.dN == full.dN


def test_violations_bruteforce():
    rnd = random.Random(5)
    for seed in range(6):
        g = G(gg.random_small(30, 0.2, seed))
        W = _dense(g)
        C = [rnd.randrange(5) for _ in range(g.n)]
        bad = 0
        for i in range(g.n):
            cand = defaultdict(float)
            for j in np.nonzero(W[i])[0]:
                if j != i:
                    cand[C[j]] += W[i, j]
            if cand and cand.get(C[i], 0.0) < max(cand.values()):
                bad += 1
        assert oracle.violations(g, C) == bad


def test_label_weights_definition():
    g = G(gg.random_small(20, 0.5, 9, self_loops=True))
    C = [v % 4 for v in range(g.n)]
    W = _dense(g)
    for i in range(g.n):
        ref = defaultdict(float)
        for j in np.nonzero(W[i])[0]:
            if j != i:
                ref[C[j]] += W[i, j]
        assert oracle.label_weights(g, C, i) == dict(ref)


def test_empty_and_isolated():
    """n = 0 runs no iteration; isolated and self-loop-only vertices keep their label
    and never count as moved."""
    g0 = oracle.Graph(np.zeros(1, np.int64), np.zeros(0, np.int32), None)
    r0 = oracle.lpa_sync(g0)
    assert r0.iterations == 0 and r0.dN == []
    g = G(gg.from_edges(4, [(0, 0), (1, 2)]))      # 0: self-loop only, 3: isolated
    r = oracle.lpa_sync(g, 0.05, 20, 4)
    assert r.labels.tolist() == [0, 1, 1, 3]
    assert r.dN == [1, 0]


def test_sweep_window_equals_first_sync_sweep():
    """One all-active sweep on a window of rows equals the first iteration of the
    synchronous run restricted to that window (used for sampled baselines)."""
    csr = gg.rmat(12, weights="int8")
    g = G(csr)
    r1 = oracle.lpa_sync(g, 0.05, 1, 4)              # l = 0 is a Pick-Less sweep
    labels0 = np.arange(g.n, dtype=np.int32)
    for v0, v1 in [(0, 1), (0, 300), (1000, 1777), (g.n - 50, g.n)]:
        out, e = oracle.sweep_window(v0, v1, g.off[v0:v1 + 1], g.idx[g.off[v0]:g.off[v1]],
                                     g.w[g.off[v0]:g.off[v1]], labels0, pl=True)
        assert out.tolist() == r1.labels[v0:v1].tolist()
        assert e == g.off[v1] - g.off[v0]
        out2, _ = oracle.sweep_range(g, labels0, v0, v1, pl=True)
        assert out2.tolist() == out.tolist()


# ---------------------------------------------------------------------------------------
# the multicore CPU baseline gives the oracle's synchronous result

@pytest.mark.parametrize("seed", range(4))
def test_multicore_baseline_equals_oracle(seed):
    import random
    rnd = random.Random(seed)
    csr = gg.random_small(rnd.choice([60, 200, 400]), rnd.choice([0.02, 0.1]), 500 + seed, wmax=rnd.choice([1, 5]),
                          self_loops=seed % 2 == 1)
    og = oracle.Graph.of(csr)
    for pl in (0, 4):
        ref = oracle.lpa_sync(og, 0.05, 20, pl)
        for threads in (1, 3):
            got = oracle.multicore_lpa_sync(og, 0.05, 20, pl, threads=threads)
            assert got.labels.tolist() == ref.labels.tolist()
            assert got.dN == ref.dN and got.iterations == ref.iterations
            assert got.active.tolist() == ref.active.tolist()
            assert got.edges == ref.edges


def test_multicore_baseline_rmat_and_closed_forms():
    for csr in (gg.rmat(11, weights="int8"), gg.complete_bipartite(6), gg.two_cliques_bridge(7), gg.star(12)):
        og = oracle.Graph.of(csr)
        ref = oracle.lpa_sync(og, 0.05, 20, 4)
        got = oracle.multicore_lpa_sync(og, 0.05, 20, 4, threads=4)
        assert got.labels.tolist() == ref.labels.tolist() and got.dN == ref.dN


# ---------------------------------------------------------------------------------------
# Cross-Check (Section 4.1): closed forms, order of the checks, dense restatement

def _dense_sync_cc(W, tol, max_iters, pl_period, cc_period):
    """_dense_sync with the Cross-Check after every cc_period-th sweep: moved vertices are
    checked in increasing id order; a move of i to c is kept when vertex c holds label c at
    that moment (earlier reverts included), else i goes back to its label before the sweep."""
    n = W.shape[0]
    C = list(range(n))
    act = [True] * n
    dns, per_iter = [], []
    for l in range(max_iters):
        pl = pl_period > 0 and l % pl_period == 0
        Cn, an, ch = list(C), [False] * n, 0
        for i in range(n):
            if not act[i]:
                continue
            c = _best_dense(W, C, i)
            if c is not None and c != C[i] and (not pl or c < C[i]):
                Cn[i] = c
                ch += 1
                for j in np.nonzero(W[i])[0]:
                    an[j] = True
        if cc_period > 0 and l % cc_period == 0:
            for i in range(n):
                if Cn[i] != C[i] and Cn[Cn[i]] != Cn[i]:
                    Cn[i] = C[i]
                    ch -= 1
        C, act = Cn, an
        dns.append(ch)
        per_iter.append(list(C))
        if not pl and ch / n < tol:
            break
    return dns, per_iter


def test_cross_check_breaks_the_bipartite_swap():
    """K_{n,n} without Pick-Less, Cross-Check after every sweep.  Sweep 0: every A vertex
    (ids 0..n-1) picks label n, every B vertex label 0.  In id order A checks first: vertex n
    still holds 0, not n, so every A move is reverted; then each B vertex finds vertex 0 back
    in community 0 and keeps its move (n moves remain).  Sweep 1: A vertices 1..n-1 join 0
    (vertex 0 keeps it, B already holds 0; n-1 moves, all good).  Sweep 2: no move, the run
    converges after 3 sweeps with one community.  Without the check the swap repeats to the
    cap."""
    for n in (2, 3, 6):
        g = G(gg.complete_bipartite(n))
        r = oracle.lpa_sync(g, 0.05, 20, 0, cc_period=1)
        assert r.dN == [n, n - 1, 0] and r.iterations == 3 and r.converged
        assert set(r.labels.tolist()) == {0}
        swap = oracle.lpa_sync(g, 0.05, 20, 0)
        assert swap.iterations == 20 and not swap.converged


def test_cross_check_order_on_a_path():
    """Path 0-1-...-(k-1), Pick-Less and Cross-Check after sweep 0.  Every vertex but 0
    picks its left neighbour's label (a tie broken by the smaller label).  Checked in id
    order: 1 keeps 0 (vertex 0 holds 0); 2 reverts (vertex 1 now holds 0, not 1); 3 keeps 2
    (vertex 2 is back at 2); 4 reverts; ...: odd vertices keep, even ones revert.  (Checking
    all moves against the labels after the sweep at once would revert every vertex but 1.)"""
    for k in (2, 5, 8, 11):
        g = G(gg.from_edges(k, [(i, i + 1) for i in range(k - 1)]))
        r = oracle.lpa_sync(g, 0.0, 1, 1, cc_period=1)
        assert r.labels.tolist() == [i - (i % 2) for i in range(k)]
        assert r.dN == [k // 2]


def test_cross_check_function_by_hand():
    C, k = oracle.cross_check([1, 0, 2, 2], [0, 1, 2, 3])     # a swap 0 <-> 1 and 3 joining 2
    assert C.tolist() == [0, 0, 2, 2] and k == 1                # 0 reverts, then 1 keeps 0


@pytest.mark.parametrize("seed", range(12))
def test_sync_cross_check_matches_dense_restatement(seed):
    rnd = random.Random(300 + seed)
    n = rnd.randint(5, 64)
    g = G(gg.random_small(n, rnd.choice([0.05, 0.1, 0.3]), 900 + seed, wmax=rnd.choice([1, 4]),
                          self_loops=(seed % 3 == 0)))
    W = _dense(g)
    pl, cc = rnd.choice([(0, 1), (0, 2), (4, 1), (2, 2), (3, 4)])
    dns, per_iter = _dense_sync_cc(W, 0.05, 20, pl, cc)
    r = oracle.lpa_sync(g, 0.05, 20, pl, cc_period=cc)
    assert r.dN == dns and r.labels.tolist() == per_iter[-1]
    for t in range(1, len(per_iter) + 1):
        assert oracle.lpa_sync(g, 0.05, t, pl, cc_period=cc).labels.tolist() == per_iter[t - 1]


def test_tolerance_test_is_strict_and_skips_pick_less_sweeps():
    """Algorithm 1 stops after a non-Pick-Less sweep l with dN_l / N < tolerance (strictly, in
    double): a tolerance equal to a sweep's ratio does not stop at that sweep, the next double
    above it does, and a Pick-Less sweep never stops the loop."""
    g = G(gg.rmat(11, weights="int8"))
    n, pl = g.n, 4
    base = oracle.lpa_sync(g, 0.0, 20, pl)             # tolerance 0: only the cap stops it
    ratios = [(l, base.dN[l] / n) for l in range(base.iterations) if l % pl != 0]
    k = next(l for i, (l, r) in enumerate(ratios) if i > 0 and 0 < r < min(x for _, x in ratios[:i]))
    tau = base.dN[k] / n
    eq = oracle.lpa_sync(g, tau, 20, pl)
    up = oracle.lpa_sync(g, float(np.nextafter(tau, 1.0)), 20, pl)
    assert eq.converged and eq.iterations > k + 1 and eq.dN == base.dN[:eq.iterations]
    assert up.converged and up.iterations == k + 1 and up.dN == base.dN[:k + 1]
    big = oracle.lpa_sync(g, 1.0, 20, pl)              # sweep 0 is Pick-Less: only sweep 1 stops
    assert big.converged and big.iterations == 2
    assert oracle.lpa_sync(g, 1.0, 20, 0).iterations == 1
    for tol, its in ((tau, eq.iterations), (float(np.nextafter(tau, 1.0)), k + 1)):
        mc = oracle.multicore_lpa_sync(g, tol, 20, pl)
        assert mc.iterations == its and mc.dN == base.dN[:its]


# --------------------------------------------------------------------------------------
# the asynchronous mode under a wave schedule (a reading of Section 4 item 1 for a parallel
# sweep: each wave reads the state at its start, its moves and marks land at its end)

def _dense_waves(W, wave_of, tol, max_iters, pl_period, take_of=None):
    """Dense restatement: per sweep, per wave in increasing index, the vertices whose take wave
    it is read and clear their flags; then the flagged vertices deciding in the wave decide on
    the labels frozen at its start, then the wave's moves and marks apply."""
    n = W.shape[0]
    take_of = wave_of if take_of is None else take_of
    C = list(range(n))
    act = [True] * n
    dns = []
    for l in range(max_iters):
        pl = pl_period > 0 and l % pl_period == 0
        ch = 0
        taken = [False] * n
        for q in range(max(wave_of) + 1):
            for i in range(n):
                if take_of[i] == q:
                    taken[i] = act[i]
                    act[i] = False
            frozen = list(C)
            members = [i for i in range(n) if wave_of[i] == q and taken[i]]
            moves = []
            for i in members:
                c = _best_dense(W, frozen, i)
                if c is not None and c != frozen[i] and (not pl or c < frozen[i]):
                    moves.append((i, c))
            for i, c in moves:
                C[i] = c
                ch += 1
                for j in np.nonzero(W[i])[0]:
                    act[j] = True
        dns.append(ch)
        if not pl and ch / n < tol:
            break
    return dns, C, act


@pytest.mark.parametrize("seed", range(12))
def test_async_waves_match_dense_restatement(seed):
    rnd = random.Random(700 + seed)
    n = rnd.randint(5, 64)
    g = G(gg.random_small(n, rnd.choice([0.05, 0.15, 0.3]), 900 + seed, wmax=rnd.choice([1, 8]),
                          self_loops=(seed % 3 == 0)))
    W = _dense(g)
    n_waves = rnd.choice([1, 2, 3, 7, n])
    wave_of = [rnd.randrange(n_waves) for _ in range(n)]
    wave_of[0] = n_waves - 1                      # every index below the largest is allowed to stay empty
    tol, mi, pl = rnd.choice([0.0, 0.05]), rnd.choice([5, 20]), rnd.choice([0, 2, 4])
    dns, C, act = _dense_waves(W, wave_of, tol, mi, pl)
    r = oracle.lpa_async_waves(g, wave_of, tol, mi, pl)
    assert r.dN == dns
    assert r.labels.tolist() == C
    assert r.active.astype(bool).tolist() == act


@pytest.mark.parametrize("seed", range(6))
def test_async_waves_endpoints(seed):
    """One vertex per wave in id order is the sequential asynchronous run; one wave holding
    every vertex is the synchronous run (labels, dN, flags, stop)."""
    rnd = random.Random(800 + seed)
    csr = [gg.sbm(500, 25, 8, 2, seed=seed, weights="int8"), gg.rmat(9, weights="int8"),
           gg.two_cliques_bridge(6), gg.complete_bipartite(5), gg.star(9),
           gg.random_small(200, 0.05, seed, self_loops=True)][seed]
    g = G(csr)
    pl = rnd.choice([0, 4])
    a = oracle.lpa_async(g, 0.05, 20, pl)
    w1 = oracle.lpa_async_waves(g, np.arange(g.n), 0.05, 20, pl)
    assert (a.dN, a.labels.tolist(), a.active.tolist(), a.iterations, a.converged) == \
        (w1.dN, w1.labels.tolist(), w1.active.tolist(), w1.iterations, w1.converged)
    s = oracle.lpa_sync(g, 0.05, 20, pl)
    w0 = oracle.lpa_async_waves(g, np.zeros(g.n, np.int32), 0.05, 20, pl)
    assert (s.dN, s.labels.tolist(), s.active.tolist(), s.iterations, s.converged) == \
        (w0.dN, w0.labels.tolist(), w0.active.tolist(), w0.iterations, w0.converged)


def test_async_waves_bipartite_by_hand():
    """K_{n,n}, A = 0..n-1 in wave 0 and B = n..2n-1 in wave 1, no Pick-Less.  Sweep 0:
    wave A sees only B labels, each once, and takes the smallest, n (all n move); wave B then
    sees label n on all of A and takes it, except vertex n, which holds n already: dN =
    2n - 1.  Sweep 1 (every vertex marked by a mover of the other side): every vertex sees
    only label n, its own: dN = 0 < tolerance, stop.  All labels n, Q = 0.  (The synchronous
    run swaps A and B at every sweep.)"""
    n = 5
    g = G(gg.complete_bipartite(n))
    r = oracle.lpa_async_waves(g, [0] * n + [1] * n, 0.05, 20, 0)
    assert r.dN == [2 * n - 1, 0]
    assert r.labels.tolist() == [n] * (2 * n)
    assert r.converged
    assert oracle.modularity(g, r.labels) == 0.0
    s = oracle.lpa_sync(g, 0.05, 20, 0)
    assert s.dN == [2 * n] * 20


def test_async_waves_rejects_bad_wave_index():
    g = G(gg.star(4))
    with pytest.raises(ValueError):
        oracle.lpa_async_waves(g, [0, 1, -1, 0, 0])


# --------------------------------------------------------------------------------------
# scanned-entry counts reported per sweep (the CPU baselines' unit of work)

@pytest.mark.parametrize("seed", range(4))
def test_sync_edges_are_the_rows_of_the_active_vertices(seed):
    """Synchronous sweep l scans the rows of exactly the vertices unprocessed at its start:
    stepping one sweep at a time from the saved state, sum(D_i over active i) is edges[l]."""
    g = G(gg.random_small(300, 0.03, 40 + seed, wmax=4, self_loops=seed % 2 == 0))
    deg = np.diff(g.off)
    full = oracle.lpa_sync(g, 0.02, 20, 4)
    C, A = None, None
    for t in range(1, full.iterations + 1):
        act = np.ones(g.n, bool) if A is None else A.astype(bool)
        r = oracle.lpa_sync(g, 0.02, t, 4, labels=C, active=A, start_iter=t - 1)
        assert r.edges == [int(deg[act].sum())]
        C, A = r.labels, r.active
    assert len(full.edges) == full.iterations


def test_async_edges_by_hand():
    """Five disjoint K_6 (ids contiguous), sequential asynchronous mode, Pick-Less at sweep 0.
    Sweep 0 processes all 30 vertices (150 entries): in each clique the minimum m sees larger
    labels only and is blocked; m+1..m+5 move to m in turn, each marking its clique, so every
    vertex but m+5 ends flagged.  Sweep 1 processes 5 vertices per clique (125 entries),
    none moves, and the run stops.  The synchronous run re-processes all 30 (150)."""
    g = G(gg.cliques(5, 6))
    a = oracle.lpa_async(g, 0.05, 20, 4)
    assert a.dN == [25, 0] and a.edges == [150, 125]
    assert oracle.lpa_sync(g, 0.05, 20, 4).edges == [150, 150]
    assert oracle.lpa_async_waves(g, np.arange(g.n), 0.05, 20, 4).edges == [150, 125]


@pytest.mark.parametrize("seed", range(10))
def test_async_waves_with_early_flag_takes_match_dense_restatement(seed):
    """Flags taken at an earlier wave than the decision (as when a warp fetches the flags of a
    batch before deciding its vertices one step at a time): labels, dN and flags equal an
    independent dense restatement; taking each flag in its own deciding wave is the default."""
    rnd = random.Random(1700 + seed)
    n = rnd.randint(5, 48)
    g = G(gg.random_small(n, rnd.choice([0.08, 0.2, 0.35]), 1900 + seed, wmax=rnd.choice([1, 6]),
                          self_loops=(seed % 4 == 1)))
    W = _dense(g)
    n_waves = rnd.choice([2, 3, 6, n])
    wave_of = [rnd.randrange(n_waves) for _ in range(n)]
    wave_of[0] = n_waves - 1
    take_of = [rnd.randint(0, w) for w in wave_of]
    tol, mi, pl = rnd.choice([0.0, 0.05]), rnd.choice([6, 20]), rnd.choice([0, 2, 4])
    dns, C, act = _dense_waves(W, wave_of, tol, mi, pl, take_of)
    r = oracle.lpa_async_waves(g, wave_of, tol, mi, pl, take_of=take_of)
    assert r.dN == dns
    assert r.labels.tolist() == C
    assert r.active.astype(bool).tolist() == act
    same = oracle.lpa_async_waves(g, wave_of, tol, mi, pl, take_of=wave_of)
    plain = oracle.lpa_async_waves(g, wave_of, tol, mi, pl)
    assert (same.dN, same.labels.tolist(), same.edges) == (plain.dN, plain.labels.tolist(), plain.edges)


def test_async_waves_early_take_by_hand():
    """One edge {0, 1}, no Pick-Less; vertex 0 decides in wave 0, vertex 1 in wave 1.
    Flags taken in the deciding wave: sweep 0 moves 0 to label 1, which marks 1; vertex 1 then
    takes its flag (set, cleared), sees label 1 (its own) and stays: dN = [1], no flag left, so
    sweep 1 processes nothing (edges [2, 0]).  Both flags taken at wave 0: vertex 1 takes its
    flag before vertex 0's mark lands, so the mark survives, and sweep 1 processes vertex 1
    again (edges [2, 1]); labels and dN are the same."""
    g = G(gg.from_edges(2, [(0, 1)]))
    a = oracle.lpa_async_waves(g, [0, 1], 0.05, 20, 0)
    b = oracle.lpa_async_waves(g, [0, 1], 0.05, 20, 0, take_of=[0, 0])
    assert a.dN == [1, 0] and a.edges == [2, 0] and a.labels.tolist() == [1, 1]
    assert b.dN == [1, 0] and b.edges == [2, 1] and b.labels.tolist() == [1, 1]
    with pytest.raises(ValueError):
        oracle.lpa_async_waves(g, [0, 1], take_of=[1, 1])        # a take after the decision
