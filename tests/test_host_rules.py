"""Rules the library applies at creation, restated on the CPU and checked against their direct
definitions (no GPU): the test that every CSR row's indices strictly increase, which lets a
fresh synchronous run's first sweep skip the label tables (every neighbour label is then a
distinct vertex id, so each label's sum is the one entry's weight)."""
import numpy as np
import pytest


def strict_by_descents(off, idx):
    """The creation check: count adjacent index pairs that do not increase over the whole index
    array, and those whose second entry starts a non-empty row; every row strictly increases
    iff the two counts are equal."""
    m = idx.size
    d_all = int(np.count_nonzero(idx[:-1] >= idx[1:])) if m > 1 else 0
    d_row = 0
    for i in range(1, off.size - 1):
        b, b1 = off[i], off[i + 1]
        if 0 < b < m and b1 > b and idx[b - 1] >= idx[b]:
            d_row += 1
    return d_all == d_row


def strict_by_rows(off, idx):
    return all(np.all(np.diff(idx[off[i]:off[i + 1]]) > 0) for i in range(off.size - 1))


def random_csr(rng, n, strict):
    deg = rng.integers(0, 6, size=n)
    deg[rng.random(n) < 0.3] = 0                     # empty rows, also at both ends
    rows = []
    for i in range(n):
        d = int(min(deg[i], n))
        row = np.sort(rng.choice(n, size=d, replace=False))
        rows.append(row)
    if not strict:
        cand = [i for i in range(n) if rows[i].size >= 1]
        if not cand:
            rows[0], cand = np.array([0]), [0]
        i = int(rng.choice(cand))
        kind = rng.integers(0, 3)
        if kind == 0 and rows[i].size >= 2:            # two entries out of order
            j = int(rng.integers(0, rows[i].size - 1))
            rows[i][[j, j + 1]] = rows[i][[j + 1, j]]
        elif kind == 1:                                # a repeated neighbour
            j = int(rng.integers(0, rows[i].size))
            rows[i] = np.sort(np.append(rows[i], rows[i][j]))
        else:                                          # a repeated neighbour, rows unsorted
            rows[i] = np.append(rows[i], rows[i][0])
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([r.size for r in rows])
    idx = np.concatenate(rows).astype(np.int64) if off[-1] else np.zeros(0, dtype=np.int64)
    return off, idx


@pytest.mark.parametrize("seed", range(40))
def test_strict_rows_by_descent_counts(seed):
    rng = np.random.default_rng(seed)
    for strict in (True, False):
        off, idx = random_csr(rng, int(rng.integers(1, 30)), strict)
        assert strict_by_descents(off, idx) == strict_by_rows(off, idx)


def test_strict_rows_edge_cases():
    cases = [
        ([0], []),                                     # no vertices
        ([0, 0, 0], []),                               # no entries
        ([0, 1], [0]),                                 # a self-loop
        ([0, 2, 2, 4], [0, 1, 0, 1]),                  # a row start below its predecessor
        ([0, 2, 4], [0, 1, 2, 3]),                     # a row start above its predecessor
        ([0, 2, 4], [0, 1, 1, 2]),                     # equal across a row boundary
        ([0, 2, 4], [1, 1, 0, 2]),                     # a repeat inside a row
        ([0, 0, 3, 3], [2, 1, 0]),                     # descending inside one row
    ]
    for off, idx in cases:
        off, idx = np.asarray(off, dtype=np.int64), np.asarray(idx, dtype=np.int64)
        assert strict_by_descents(off, idx) == strict_by_rows(off, idx), (off, idx)
