"""Example 2 (Sec. 3.2): the free Wilson-Dirac matrix, pinned to the paper's Tables 3-5.

The generator (Eqs. disDirac and explicit) must give the printed rank and nonzero
count; the momentum-space closed form of L^-1 must give the printed exact traces and
agree block by block with a dense inverse; the oracle's CC estimate must land on the
exact trace within its standard error.
"""
import os

import numpy as np
import pytest

import oracle
from paper_cs_0412107_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dirac_tables.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, N, val = line.split()[:3]
                out[(key, int(N))] = float(val)
    return out


def test_gamma_matrices_are_a_euclidean_clifford_set():
    g = wl.DIRAC_GAMMA
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2 * np.eye(4) * (a == b))


@pytest.mark.parametrize("N", [18, 20])
def test_table3_rank_and_nonzeros(N):
    t = _golden()
    c = wl.wilson_dirac((N,) * 4, 0.1)
    assert c.n == t[("rank", N)] and c.nnz == t[("nonzeros", N)]
    assert np.all(np.diff(c.row_ptr) == 14)
    assert np.all(c.val[c.col == np.repeat(np.arange(c.n), 14)] == 1.0)  # unit diagonal


@pytest.mark.parametrize("N", [18, 20])
def test_exact_trace_matches_tables_4_and_5(N):
    t = _golden()
    tr = wl.wilson_dirac_inverse_trace((N,) * 4, 0.1)
    assert abs(tr.imag) < 1e-6
    assert abs(tr.real - t[("exact_trace", N)]) <= 1e-7 * t[("exact_trace", N)]


def test_propagator_blocks_match_the_dense_inverse():
    """Every offset class, both directions: a swapped hop direction, a gamma on the wrong
    axis or a wrong spinor index in the generator changes one of these blocks."""
    dims = (3, 3, 3, 4)
    c = wl.wilson_dirac(dims, 0.13)
    inv = np.linalg.inv(c.to_dense())
    V = int(np.prod(dims))

    def idx(x, s):
        return x[0] + dims[0] * (x[1] + dims[1] * (x[2] + dims[2] * (x[3] + dims[3] * s)))

    x = (1, 2, 0, 3)
    for r in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (0, 0, 0, 3),
              (2, 0, 0, 0), (1, 1, 0, 0), (0, 2, 1, 2), (1, 1, 1, 1)]:
        y = tuple((x[k] + r[k]) % dims[k] for k in range(4))
        blk = np.array([[inv[idx(x, s), idx(y, u)] for u in range(4)] for s in range(4)])
        assert np.abs(blk - wl.wilson_dirac_propagator(dims, 0.13, r)).max() < 1e-13, r
    assert abs(np.trace(inv) - wl.wilson_dirac_inverse_trace(dims, 0.13)) < 1e-10 * V


def test_stop_rule_of_tables_4_and_5_is_relative_error_1e_5():
    """Both Example 2 runs stopped with SE / |estimate| just under 1e-5 (Sec. 3.1's rule
    with tol 1e-5, checked every 100 cycles)."""
    t = _golden()
    for N in (18, 20):
        rel = t[("cc_se", N)] / t[("cc_trace", N)]
        assert 0.99e-5 < rel < 1e-5


def test_oracle_trace_estimate_on_a_small_lattice():
    dims = (3, 3, 3, 3)
    c = wl.wilson_dirac(dims, 0.1)
    exact = wl.wilson_dirac_inverse_trace(dims, 0.1).real
    K, burn, samp = 32, 40, 160
    series = []
    oracle.run(c, K, seed=5, ncycles=burn + samp, acc_from=burn, q=np.ones(c.n), series_out=series)
    g = oracle.geyer_ims(np.array(series))
    assert abs(g["mean"] - exact) < 4 * g["se"]
    assert g["se"] < 0.01 * exact


def test_spin_fastest_numbering_is_a_relabelling():
    """The spinor-fastest numbering is P L P^T of the paper's spinor-slowest one."""
    dims = (3, 3, 3, 4)
    V = int(np.prod(dims))
    a = wl.wilson_dirac(dims, 0.1).to_dense()
    b = wl.wilson_dirac(dims, 0.1, spin_fastest=True).to_dense()
    i = np.arange(4 * V)
    new = (i % V) * 4 + i // V  # row i = site + V s of the paper's numbering -> 4 site + s
    assert np.array_equal(b[np.ix_(new, new)], a)
