"""Small shared helpers for the tests (no solver arithmetic)."""
import os
from dataclasses import dataclass

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@dataclass
class CSR:
    m: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self):
        return int(self.row_ptr[-1])

    def dense(self):
        a = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        a[rows, self.col] = self.val
        return a


def csr_from_dense(a):
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    rows, cols = np.nonzero(a)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(m, n, row_ptr, cols.astype(np.int32), a[rows, cols].copy())


def read_golden_rows(name):
    """Numeric rows of a golden file; '#' lines are comments and separate blocks."""
    blocks, cur = [], []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                if cur:
                    blocks.append(cur)
                    cur = []
                continue
            cur.append(line.split())
    if cur:
        blocks.append(cur)
    return blocks


def random_sparse(m, n, per_row, rng, scale_exp=0.0):
    """Random CSR with `per_row` distinct columns per row and column scaling 10^(-scale_exp j/(n-1))."""
    cols = np.stack([np.sort(rng.choice(n, per_row, replace=False)) for _ in range(m)])
    vals = rng.standard_normal((m, per_row)) * (10.0 ** (-scale_exp * np.arange(n) / max(n - 1, 1)))[cols]
    row_ptr = np.arange(m + 1, dtype=np.int64) * per_row
    return CSR(m, n, row_ptr, cols.reshape(-1).astype(np.int32), vals.reshape(-1))
