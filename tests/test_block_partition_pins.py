"""The block partition of Sec. 4, pinned on the FP64 oracle: small non-singular
diagonal blocks D_b around zeros of the diagonal, each block updated as a whole
with A_b B_b^H = D_b^-1 (the block form of the demonstration of Sec. 2.2)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_cs_0412107_gb300 import workloads as wl


def zero_diagonal_pairs(npairs, seed, complex_=False, coupling=0.12):
    """Rows (2k, 2k+1) form a block [[0, a], [b, 0]] with ab < 0 (a zero diagonal, so the
    scalar sweep cannot run; eigenvalues +-i sqrt|ab|, so the block has a real principal
    square root), plus weak random couplings between blocks."""
    rng = np.random.default_rng(seed)
    n = 2 * npairs
    rows, cols, vals = [], [], []
    for k in range(npairs):
        i = 2 * k
        sgn = rng.choice([-1, 1])
        a, b = rng.uniform(1.0, 2.0) * sgn, -rng.uniform(1.0, 2.0) * sgn
        rows += [i, i + 1]; cols += [i + 1, i]; vals += [a, b]
    for i in range(n):
        for j in rng.choice(n, 3, replace=False):
            if j // 2 != i // 2:
                v = coupling * rng.uniform(-1, 1)
                if complex_:
                    v = v * np.exp(1j * rng.uniform(0, 2 * np.pi))
                rows.append(i); cols.append(j); vals.append(v)
    vals = np.array(vals, dtype=np.complex128 if complex_ else np.float64)
    return wl.csr_from_coo(n, rows, cols, vals), np.arange(0, n + 1, 2)


def test_one_row_blocks_are_the_scalar_sweep():
    c = wl.random_dominant(40, 4, 1.4, 2)
    st_b = oracle.run_block(c, np.arange(c.n + 1), 16, seed=3, ncycles=12)
    st_s, _, _ = oracle.run(c, 16, seed=3, ncycles=12)
    assert np.abs(st_b.z - st_s.z).max() < 1e-12 * np.abs(st_s.z).max()
    assert np.abs(st_b.w - st_s.w).max() < 1e-12 * np.abs(st_s.w).max()


@pytest.mark.parametrize("complex_", [False, True])
def test_enumerated_expectation_is_the_block_recursion(complex_):
    """Every noise history of two cycles on n = 4 (2^8 of them, one per chain): the exact
    mean of z w^H equals the expected-covariance recursion with block D."""
    c, _ = zero_diagonal_pairs(2, 5, complex_, coupling=0.3)
    bp = np.array([0, 2, 4])
    a = c.to_dense().astype(np.complex128)
    n, cycles = 4, 2
    hist = np.array(list(itertools.product([1.0, -1.0], repeat=n * cycles))).T  # [n*cycles][256]
    fac = oracle.block_factors(c, bp)
    st = oracle.State(n, hist.shape[1])
    for k in range(cycles):
        oracle.block_cycle(a, fac, st, hist[k * n:(k + 1) * n])
    emp = st.z @ st.w.conj().T / hist.shape[1]
    assert np.abs(emp - oracle.block_expected_covariance(a, bp, cycles)).max() < 1e-12


def test_block_recursion_fixed_point_is_the_inverse():
    c, bp = zero_diagonal_pairs(6, 7, True)
    a = c.to_dense()
    assert np.abs(oracle.block_expected_covariance(a, bp, 400) - np.linalg.inv(a)).max() < 1e-10


def test_block_factors_satisfy_the_condition():
    c, bp = zero_diagonal_pairs(5, 8, True)
    a = c.to_dense().astype(np.complex128)
    for r, Dinv, A, B in oracle.block_factors(c, bp):
        assert np.abs(A @ B.conj().T - Dinv).max() < 1e-12


@pytest.mark.parametrize("complex_", [False, True])
def test_block_sweep_estimates_the_inverse_where_the_scalar_one_cannot_start(complex_):
    c, bp = zero_diagonal_pairs(30, 11, complex_)
    with pytest.raises(ValueError):
        oracle.row_constants(c)  # zero diagonal: Eqs. 4/5 cannot run
    inv = np.linalg.inv(c.to_dense())
    K, G, burn, samp = 256, 32, 40, 200
    st = oracle.run_block(c, bp, K, seed=4, ncycles=burn)
    acc = np.zeros((c.n, c.n, G), dtype=np.complex128)
    for k in range(samp):
        st = oracle.run_block(c, bp, K, seed=4, cycle0=burn + k, ncycles=1, state=st)
        for g in range(G):
            sl = slice(g * K // G, (g + 1) * K // G)
            acc[:, :, g] += st.z[:, sl] @ st.w[:, sl].conj().T
    gm = acc / (samp * K // G)
    mean = gm.mean(axis=2)
    se = np.sqrt(((gm.real - mean.real[:, :, None]) ** 2).sum(axis=2) / (G * (G - 1)))
    z = np.abs(mean.real - inv.real) / np.maximum(se, 1e-12)
    assert (z > 3).mean() < 0.01 and 0.8 < np.sqrt(np.mean(z ** 2)) < 1.25


def test_hermitian_blocks_give_w_equal_z():
    c, bp = zero_diagonal_pairs(4, 2, True)
    a = c.to_dense()
    h = (a + a.conj().T) / 2
    h[np.diag_indices(c.n)] = 0
    for k in range(0, c.n, 2):  # Hermitian positive-definite 2x2 blocks
        h[k, k], h[k + 1, k + 1] = 3.0, 2.5
    hc = wl.csr_from_coo(c.n, *np.nonzero(h), h[np.nonzero(h)])
    st = oracle.run_block(hc, bp, 8, seed=1, ncycles=10)
    assert np.abs(st.z - st.w).max() < 1e-12 * np.abs(st.z).max()


def test_block_without_principal_square_root_is_rejected():
    c = wl.csr_from_coo(2, [0, 1], [1, 0], np.array([1.0, 2.0]))  # eigenvalues +-sqrt(2)
    with pytest.raises(ValueError):
        oracle.block_factors(c, np.array([0, 2]))

