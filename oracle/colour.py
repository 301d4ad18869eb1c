"""The colour sweep order of Sec. 4 (reordering the rows and columns of C),
written out from its definition for the oracle's use: rows, in ascending order,
take the smallest colour not used by an already-coloured neighbour in the
graph of C + C^T; the order lists colour 0's rows ascending, then colour 1's,
and so on.  ``permuted`` forms C' = P C P^T, the matrix a colour-ordered
sampler runs on (its chains follow the oracle on C').

TEST INFRASTRUCTURE, like the rest of this package.
"""
from __future__ import annotations

import numpy as np


class CSR:
    """A CSR matrix as the oracle reads it: n, row_ptr int64[n+1], col int32[nnz], val."""

    def __init__(self, n, row_ptr, col, val):
        self.n = int(n)
        self.row_ptr = row_ptr
        self.col = col
        self.val = val

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def _lower_neighbours(csr):
    n = csr.n
    rows = np.repeat(np.arange(n), np.diff(csr.row_ptr))
    col = np.asarray(csr.col, dtype=np.int64)
    off = col != rows
    a = np.concatenate([rows[off], col[off]])
    b = np.concatenate([col[off], rows[off]])
    keep = b < a  # neighbours coloured before the row
    a, b = a[keep], b[keep]
    o = np.argsort(a, kind="stable")
    return np.searchsorted(a[o], np.arange(n + 1)), b[o]


def greedy_order(csr):
    """Returns (order, colour of each row)."""
    ptr, nb = _lower_neighbours(csr)
    color = np.zeros(csr.n, dtype=np.int64)
    for i in range(csr.n):
        used = set(color[nb[ptr[i]:ptr[i + 1]]].tolist())
        k = 0
        while k in used:
            k += 1
        color[i] = k
    order = np.lexsort((np.arange(csr.n), color))
    return order.astype(np.int64), color


def permuted(csr, order):
    """C' = P C P^T: row k of C' is row order[k] of C (columns renumbered the same way,
    sorted within each row)."""
    n = csr.n
    inv = np.empty(n, dtype=np.int64)
    inv[order] = np.arange(n)
    rows = inv[np.repeat(np.arange(n), np.diff(csr.row_ptr))]
    cols = inv[np.asarray(csr.col, dtype=np.int64)]
    o = np.lexsort((cols, rows))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return CSR(n, np.cumsum(row_ptr), cols[o].astype(np.int32), np.asarray(csr.val)[o])
