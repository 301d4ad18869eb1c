"""The colour sweep order written out from its definition (Sec. 4: reordering the
rows and columns of C), for the tests: rows in ascending order take the smallest
colour not used by an already-coloured neighbour in the graph of C + C^T; the
order lists colour 0's rows ascending, then colour 1's, ..."""
import numpy as np


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


def neighbours(csr):
    """Neighbour sets of every row in the graph of C + C^T."""
    nbr = [set() for _ in range(csr.n)]
    for i in range(csr.n):
        for e in range(csr.row_ptr[i], csr.row_ptr[i + 1]):
            j = int(csr.col[e])
            if j != i:
                nbr[i].add(j)
                nbr[j].add(i)
    return nbr


def permuted(csr, order):
    """C' = P C P^T: row k of C' is row order[k] of C."""
    from paper_cs_0412107_gb300 import workloads as wl
    inv = np.empty(csr.n, dtype=np.int64)
    inv[order] = np.arange(csr.n)
    rows = np.repeat(np.arange(csr.n), np.diff(csr.row_ptr))
    return wl.csr_from_coo(csr.n, inv[rows], inv[csr.col], csr.val)
