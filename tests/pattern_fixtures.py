"""Matrices with a known number of distinct column-offset tuples (the tuples
of j - i over a row's entries in CSR order), for the pattern-coded column
tests: pinned on the CPU by tests/test_pattern_fixtures.py, used on the GPU
by tests/test_gpu_patterns.py."""
import numpy as np

from paper_2303_02352_gb300 import workloads as W


def csr_from_coo(n, r, c, v):
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rp = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rp, r + 1, 1)
    return W.CSR(n, np.cumsum(rp).astype(np.int32), c.astype(np.int32), v)


def block_diagonal(sizes, periods):
    """Dense blocks k x k (diagonal k, off-diagonal -1: symmetric, strictly
    diagonally dominant), the sequence `sizes` repeated `periods` times.  Row r
    of a block of size k has the column offsets (-r, ..., k-1-r), so the matrix
    has exactly sum(set(sizes)) distinct offset tuples."""
    rows, cols, vals = [], [], []
    base = 0
    for _ in range(periods):
        for k in sizes:
            idx = np.arange(base, base + k)
            rr, cc = np.meshgrid(idx, idx, indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(np.where(rr == cc, float(k), -1.0).ravel())
            base += k
    return csr_from_coo(base, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def paired_rows(dmax, singleton, periods):
    """Rows coupled in pairs at distance d = 1 .. dmax (a block of 2d rows: row
    j with row j + d; diagonal 2, coupling -1), with one uncoupled row per
    period if `singleton`: 2 dmax (+ 1) distinct offset tuples of at most two
    entries, (0, d) and (-d, 0) (and (0,))."""
    rows, cols, vals = [], [], []
    base = 0
    for _ in range(periods):
        for d in range(1, dmax + 1):
            a = np.arange(base, base + d)
            rows += [a, a + d, a, a + d]
            cols += [a, a + d, a + d, a]
            vals += [np.full(d, 2.0), np.full(d, 2.0), np.full(d, -1.0), np.full(d, -1.0)]
            base += 2 * d
        if singleton:
            rows.append(np.array([base]))
            cols.append(np.array([base]))
            vals.append(np.array([1.0]))
            base += 1
    return csr_from_coo(base, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
