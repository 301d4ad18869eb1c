"""The colour sweep order (Sec. 4, reordering C) computed by the library on the
host: it must be the greedy colouring order of its definition, a proper colouring
of the graph of C + C^T, and give one dependency level per colour."""
import numpy as np
import pytest

from _greedy import greedy_order, neighbours, permuted
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


CASES = [lambda: wl.random_dominant(300, 4, 1.5, 3), lambda: wl.pedigree(2000, 1.2, 4),
         lambda: wl.u1_lattice((12, 10), 0.12, 0.08, seed=1), lambda: wl.u1_lattice((5, 7), 0.12, 0.08, seed=2),
         lambda: wl.wilson_dirac((3, 3, 3, 4), 0.1)]


@pytest.mark.parametrize("make", CASES)
def test_library_order_is_the_greedy_colouring(make):
    c = make()
    order, nc = mcinv.mcinv_color_order(c.n, c.row_ptr, c.col)
    want, color = greedy_order(c)
    nbr = neighbours(c)
    assert np.array_equal(order, want) and nc == color.max() + 1
    # a proper colouring: no edge of C + C^T joins two rows of one colour
    for i in range(c.n):
        assert all(color[j] != color[i] for j in nbr[i])


@pytest.mark.parametrize("make", CASES)
def test_levels_of_the_permuted_matrix_are_the_colours(make):
    """In C' = P C P^T every row's lower neighbours have a smaller colour, so the
    Gauss-Seidel dependency depth is at most the number of colours."""
    c = make()
    order, nc = mcinv.mcinv_color_order(c.n, c.row_ptr, c.col)
    cp = permuted(c, order)
    level = np.zeros(c.n, dtype=np.int64)
    rows = np.repeat(np.arange(c.n), np.diff(cp.row_ptr))
    lower = {}
    for r, j in zip(rows, cp.col):
        if j < r:
            lower.setdefault(r, []).append(j)
        elif j > r:
            lower.setdefault(j, []).append(r)
    for i in range(c.n):
        if i in lower:
            level[i] = max(level[j] for j in lower[i]) + 1
    assert level.max() + 1 <= nc


def test_even_periodic_lattices_take_two_colours():
    for c in (wl.u1_lattice((16, 12), 0.12, 0.08, seed=0), wl.u1_lattice((4, 4, 4, 4), 0.06, 0.04, seed=0),
              wl.wilson_dirac((4, 4, 4, 4), 0.1)):
        assert mcinv.mcinv_color_order(c.n, c.row_ptr, c.col)[1] == 2


def test_malformed_input_is_rejected():
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_color_order(2, [0, 1, 2], [1, 0])  # no diagonal
    assert e.value.status == mcinv.MCINV_E_SINGULAR_DIAG
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_color_order(2, [0, 1, 2], [0, 5])
    assert e.value.status == mcinv.MCINV_E_ARG
