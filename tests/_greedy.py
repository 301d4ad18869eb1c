"""The colour sweep order written out from its definition (Sec. 4: reordering the
rows and columns of C), for the tests: rows in ascending order take the smallest
colour not used by an already-coloured neighbour in the graph of C + C^T; the
order lists colour 0's rows ascending, then colour 1's, ..."""
import numpy as np

from oracle.colour import greedy_order, permuted  # noqa: F401  (the oracle's own statement)


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
