"""The colour sweep order written out from its definition (Sec. 4: reordering the
rows and columns of C), for the tests: rows in ascending order take the smallest
colour not used by an already-coloured neighbour in the graph of C + C^T; the
order lists colour 0's rows ascending, then colour 1's, ..."""
import numpy as np


def greedy_order(csr):
    n = csr.n
    nbr = [set() for _ in range(n)]
    for i in range(n):
        for e in range(csr.row_ptr[i], csr.row_ptr[i + 1]):
            j = int(csr.col[e])
            if j != i:
                nbr[i].add(j)
                nbr[j].add(i)
    color = [0] * n
    for i in range(n):
        used = {color[j] for j in nbr[i] if j < i}
        k = 0
        while k in used:
            k += 1
        color[i] = k
    order = sorted(range(n), key=lambda i: (color[i], i))
    return np.array(order, dtype=np.int64), np.array(color), nbr


def permuted(csr, order):
    """C' = P C P^T: row k of C' is row order[k] of C."""
    from paper_cs_0412107_gb300 import workloads as wl
    inv = np.empty(csr.n, dtype=np.int64)
    inv[order] = np.arange(csr.n)
    rows = np.repeat(np.arange(csr.n), np.diff(csr.row_ptr))
    return wl.csr_from_coo(csr.n, inv[rows], inv[csr.col], csr.val)
