"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these re-type the oracle's loops: each compares it with a different
statement of the same fact (published test vectors, the matrix form the paper
derives, closed forms, exact expectations by enumeration, dense inverses).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_cs_0412107_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small_random(n, seed, complex_=False, dominance=1.5, density=3):
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in rng.choice(n, size=min(density, n), replace=False):
            if j == i:
                continue
            v = rng.uniform(-1, 1)
            if complex_:
                v = v + 1j * rng.uniform(-1, 1)
            rows.append(i); cols.append(j); vals.append(v)
    vals = np.array(vals, dtype=np.complex128 if complex_ else np.float64)
    absum = np.zeros(n)
    np.add.at(absum, np.array(rows, dtype=np.int64), np.abs(vals))
    d = dominance * np.maximum(absum, 0.5)
    if complex_:
        d = d * np.exp(1j * rng.uniform(-0.6, 0.6, size=n))  # complex diagonal
    return wl.csr_from_coo(n, rows + list(range(n)), cols + list(range(n)),
                           np.concatenate([vals, d.astype(vals.dtype)]))


# -- Philox4x32-10 -----------------------------------------------------------------------

def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_noise_moments():
    """Eqs. 5a/5b: E phi = 0, E phi phi^T = I, independent across cycles and chains."""
    n, draws = 64, 600
    P = np.array([oracle.noise_matrix(n, 11, 0, c, 3) for c in range(draws)])
    assert set(np.unique(P)) == {-1.0, 1.0}
    assert np.abs(P.mean(axis=0)).max() < 5 / np.sqrt(draws)
    cov = P.T @ P / draws
    assert np.allclose(np.diag(cov), 1.0)
    off = cov - np.diag(np.diag(cov))
    assert np.abs(off).max() < 5 / np.sqrt(draws)
    Q = np.array([oracle.noise_matrix(n, 11, 0, c, 4) for c in range(draws)])
    assert np.abs((P * Q).mean(axis=0)).max() < 5 / np.sqrt(draws)
    # the noise of one chain does not depend on the matrix id only through nothing
    R = np.array([oracle.noise_matrix(n, 11, 1, c, 3) for c in range(50)])
    assert (R != P[:50]).mean() > 0.3


def test_noise_bit_layout():
    """Row r takes bit (r & 31) of word ((r >> 5) & 3) of Philox(ctr=(r>>7, chain, cycle, matrix))."""
    seed = 0x123456789ABCDEF
    for row in (0, 1, 31, 32, 95, 127, 128, 1000, 70001):
        out = oracle.philox4x32_10((row >> 7, 5, 9, 2), (seed & 0xffffffff, seed >> 32))
        bit = (out[(row >> 5) & 3] >> (row & 31)) & 1
        assert oracle.phi(seed, 2, 5, 9, row) == (-1 if bit else 1)


# -- per-row constants ----------------------------------------------------------------------

def test_row_constants_product():
    """alpha_i conj(beta_i) = 1/c_ii (needed by Eqs. Theta/Gamma/series), incl. negative reals."""
    diag = np.array([4.0, -9.0, 2.0 + 3.0j, -4.0 + 0.0j, -4.0 - 0.0j, 1e-3 - 5j], dtype=np.complex128)
    n = len(diag)
    csr = wl.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), diag)
    a, b, d = oracle.row_constants(csr)
    assert np.allclose(a * np.conj(b), 1 / diag, rtol=1e-14)
    assert np.allclose(d, 1 / diag, rtol=1e-14)
    assert np.allclose(a, 1 / np.sqrt(diag), rtol=1e-14)  # principal root, Eq. 4
    real = wl.CSR(2, np.arange(3, dtype=np.int64), np.arange(2, dtype=np.int32), np.array([4.0, -9.0]))
    a, b, d = oracle.row_constants(real)
    assert np.allclose(a.real, [0.5, 1 / 3]) and np.allclose(b.real, [0.5, -1 / 3])
    assert np.all(a.imag == 0) and np.all(b.imag == 0)


def test_singular_diagonal_rejected():
    csr = wl.CSR(2, np.array([0, 1, 2], dtype=np.int64), np.array([1, 1], dtype=np.int32),
                 np.array([1.0, 2.0]))
    with pytest.raises(ValueError, match="row 0"):
        oracle.run(csr, 2, ncycles=1)
    z = wl.CSR(2, np.array([0, 1, 2], dtype=np.int64), np.array([0, 1], dtype=np.int32),
               np.array([1.0, 0.0]))
    with pytest.raises(ValueError, match="row 1"):
        oracle.run(z, 2, ncycles=1)


# -- the sweep against its matrix form ------------------------------------------------------

@pytest.mark.parametrize("complex_", [False, True])
def test_sweep_matches_matrix_form(complex_):
    """Eqs. 4/5 element by element == Eqs. mform1/mform2 solved as triangular systems."""
    n, K, cycles, seed = 13, 3, 6, 42
    csr = _small_random(n, 5, complex_=complex_)
    a = csr.to_dense().astype(np.complex128)
    alpha, beta, _ = oracle.row_constants(csr)
    st = oracle.State(n, K)
    st.z[:] = np.random.default_rng(1).normal(size=(n, K))  # arbitrary start
    st.w[:] = np.random.default_rng(2).normal(size=(n, K))
    z = st.z.copy(); w = st.w.copy()
    oracle.run(csr, K, seed=seed, cycle0=10, ncycles=cycles, state=st, chain0=7)
    for k in range(cycles):
        for c in range(K):
            phi = oracle.noise_matrix(n, seed, 0, 7 + c, 10 + k)
            z[:, c], w[:, c] = oracle.matrix_form_step(a, alpha, beta, phi, z[:, c], w[:, c])
    assert np.abs(st.z - z).max() < 1e-12 * max(1, np.abs(z).max())
    assert np.abs(st.w - w).max() < 1e-12 * max(1, np.abs(w).max())


def test_lower_triangular_forgets_z():
    """U = 0: z^(k) = (D+L)^-1 D alpha phi^(k), whatever z^(k-1) was (Eq. zk)."""
    n = 9
    csr = _small_random(n, 3)
    a = np.tril(csr.to_dense())
    low = wl.csr_from_coo(n, *np.nonzero(a), a[np.nonzero(a)])
    alpha, _, _ = oracle.row_constants(low)
    st = oracle.State(n, 2)
    st.z[:] = 1e3
    oracle.run(low, 2, seed=3, cycle0=5, ncycles=1, state=st)
    import scipy.linalg as sl
    for c in range(2):
        phi = oracle.noise_matrix(n, 3, 0, c, 5)
        want = sl.solve_triangular(a, np.diag(np.diag(a)) @ (alpha.real * phi), lower=True)
        assert np.allclose(st.z[:, c], want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("complex_", [False, True])
def test_diagonal_matrix_exact(complex_):
    """Diagonal C: z_i = phi_i/sqrt(c_ii) and each sample z_i conj(w_i) = 1/c_ii (Sec. 4)."""
    n = 17
    rng = np.random.default_rng(0)
    d = rng.uniform(0.5, 3, n) * rng.choice([-1, 1], n)
    if complex_:
        d = d * np.exp(1j * rng.uniform(-1, 1, n))
    csr = wl.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), d)
    st, dacc, _ = oracle.run(csr, 4, seed=9, ncycles=3, acc_from=0, cpg=1)
    assert np.allclose(dacc / 3, 1 / d[None, :], rtol=1e-14)


def test_hermitian_w_equals_z():
    """Hermitian C: Eq. 5 coincides with Eq. 4 (w = z), i.e. the GS sampler of Eq. 2."""
    n = 15
    for cx in (False, True):
        b = _small_random(n, 8, complex_=cx).to_dense()
        h = b + b.conj().T
        h[np.diag_indices(n)] = np.abs(np.diag(h)).real + np.abs(h).sum(axis=1)
        csr = wl.csr_from_coo(n, *np.nonzero(h), h[np.nonzero(h)])
        st, _, _ = oracle.run(csr, 3, seed=1, ncycles=5)
        assert np.array_equal(st.z, st.w)


# -- exact expectations ---------------------------------------------------------------------

def test_expected_covariance_fixed_point_is_inverse():
    """Eq. recursive: C^-1 = (D+L)^-1 D (D+U)^-1 + T C^-1 S."""
    a = _small_random(10, 4, complex_=True).to_dense()
    assert np.allclose(oracle.expected_covariance(a, 400), np.linalg.inv(a), atol=1e-12)


def test_enumerated_expectation_matches_covariance_recursion():
    """Brute force: average z^(k) w^(k)H over every +-1 noise history (n=2, k=2)
    and compare with the exact X_k of the covariance recursion (Eqs. zn, wn, series)."""
    n, k, K, seed = 2, 2, 768, 17
    a = np.array([[2.0, -0.7 + 0.4j], [0.9 - 0.3j, 1.5 + 0.5j]])
    csr = wl.csr_from_coo(n, [0, 0, 1, 1], [0, 1, 0, 1], a.ravel())
    st, _, _ = oracle.run(csr, K, seed=seed, ncycles=k)
    keys = {}
    for c in range(K):
        pattern = tuple(oracle.phi(seed, 0, c, cyc, i) for cyc in range(k) for i in range(n))
        keys.setdefault(pattern, []).append(c)
    assert len(keys) == 2 ** (n * k)
    mean = np.zeros((n, n), dtype=np.complex128)
    for pattern, cs in keys.items():
        c = cs[0]
        for c2 in cs[1:]:  # same noise history -> bit-identical trajectory
            assert np.array_equal(st.z[:, c2], st.z[:, c]) and np.array_equal(st.w[:, c2], st.w[:, c])
        mean += np.outer(st.z[:, c], st.w[:, c].conj())
    mean /= len(keys)
    assert np.allclose(mean, oracle.expected_covariance(a, k), atol=1e-13)


def test_two_by_two_convergence_rate():
    """C = [[1,a],[b,1]]: sp(T) = |ab| (Sec. 2.2); the coupled-path difference is
    noise-free Gauss-Seidel on C d = 0 (Eq. 12) and shrinks by exactly ab per cycle."""
    for aa, bb in ((0.6, -0.9), (1.5, 1.2)):
        csr = wl.csr_from_coo(2, [0, 0, 1, 1], [0, 1, 0, 1], np.array([1.0, aa, bb, 1.0]))
        s1 = oracle.State(2, 1)
        s2 = oracle.State(2, 1)
        s2.z[:] = np.array([[1.0], [2.0]]); s2.w[:] = np.array([[1.0], [2.0]])
        prev = None
        for cyc in range(6):
            oracle.run(csr, 1, seed=4, cycle0=cyc, ncycles=1, state=s1)
            oracle.run(csr, 1, seed=4, cycle0=cyc, ncycles=1, state=s2)
            dz = (s2.z - s1.z)[1, 0]
            if prev is not None:
                assert abs(dz / prev - aa * bb) < 1e-12
            prev = dz
    # the estimate converges to [[1,-a],[-b,1]]/(1-ab) when |ab| < 1
    aa, bb = 0.6, -0.9
    csr = wl.csr_from_coo(2, [0, 0, 1, 1], [0, 1, 0, 1], np.array([1.0, aa, bb, 1.0]))
    st, dacc, bacc = oracle.run(csr, 512, seed=2, ncycles=260, acc_from=60, cpg=32,
                                R=[0, 1], S=[0, 1], diag=False)
    m, se = oracle.group_estimate(bacc, np.full(16, 32), 200)
    want = np.array([[1, -aa], [-bb, 1]]) / (1 - aa * bb)
    assert np.all(np.abs(m.real - want) < 4 * se.real + 1e-12)


def test_coupling_burnin_is_gauss_seidel():
    """Algorithm 1 steps 1-5: the coupling time equals the number of noise-free
    Gauss-Seidel sweeps (Eq. 12) taking d = (1..n) below tol, for C (z) and C^H (w)."""
    n = 30
    csr = _small_random(n, 12, complex_=True, dominance=1.3)
    a = csr.to_dense()

    def gs_count(m, tol):
        d = np.arange(1, n + 1).astype(np.complex128)
        for p in range(1, 10000):
            for i in range(n):
                d[i] = -(m[i, :i] @ d[:i] + m[i, i + 1:] @ d[i + 1:]) / m[i, i]
            if np.abs(d).max() < tol:
                return p, d
        return -1, d

    pz, _ = gs_count(a, 5e-5)
    pw, _ = gs_count(a.conj().T, 5e-5)
    p, z, w = oracle.coupling_burnin(csr, seed=5, tol=5e-5)
    assert p == max(pz, pw)


# -- statistics against a dense inverse ----------------------------------------------------------

@pytest.mark.parametrize("complex_", [False, True])
def test_estimate_within_3se_of_dense_inverse(complex_):
    """Eq. 1/C: the averaged z w^H covers C^-1 within its Monte Carlo error."""
    n, K, cpg = 20, 256, 16
    csr = _small_random(n, 21, complex_=complex_, dominance=1.4)
    R = np.arange(n)
    st, dacc, bacc = oracle.run(csr, K, seed=77, ncycles=330, acc_from=30, cpg=cpg, R=R, S=R)
    m, se = oracle.group_estimate(bacc, np.full(K // cpg, cpg), 300)
    truth = np.linalg.inv(csr.to_dense())
    zr = (m.real - truth.real) / se.real
    assert np.mean(np.abs(zr) > 3) < 0.02
    assert 0.6 < np.sqrt(np.mean(zr ** 2)) < 1.5
    if complex_:
        zi = (m.imag - truth.imag) / se.imag
        assert np.mean(np.abs(zi) > 3) < 0.02
    # the fused diagonal accumulation equals the block's diagonal
    assert np.allclose(dacc.sum(0), np.einsum("gii->i", bacc), rtol=1e-12)


def test_group_standard_error():
    rng = np.random.default_rng(3)
    G, per, samples = 40, 8, 50
    x = rng.normal(2.0, 3.0, size=(G, per * samples))
    acc = x.sum(axis=1)
    m, se = oracle.group_estimate(acc, np.full(G, per), samples)
    assert abs(m - x.mean()) < 1e-12
    assert abs(se / (3.0 / np.sqrt(G * per * samples)) - 1) < 0.35


def test_pure_gauge_lattice_closed_form():
    """Generator check: a pure-gauge U(1) lattice has diag(C^-1) = free-field closed form."""
    dims = (4, 6)
    csr = wl.u1_lattice(dims, 0.2, 0.1, seed=3, pure_gauge=True)
    inv = np.linalg.inv(csr.to_dense())
    assert np.allclose(np.diag(inv), wl.free_lattice_diag(dims, 0.2, 0.1), atol=1e-13)
    assert not np.allclose(csr.to_dense(), csr.to_dense().conj().T)  # non-Hermitian


# -- Monte Carlo error: Geyer's effective length (Sec. 2.3) ---------------------------------

def test_paper_tables_se_is_sqrt_var_over_effective_length():
    """The printed MC standard errors equal sqrt(Var / eff. length) (Tables 2, 4, 5)."""
    with open(os.path.join(GOLDEN, "paper_tables.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for r in rows:
        var, eff, se = float(r[1]), float(r[2]), float(r[3])
        assert abs(np.sqrt(var / eff) - se) <= 0.0006 * se + 5e-4


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9, -0.5])
def test_geyer_effective_length_of_ar1(rho):
    """AR(1) with coefficient rho: effective length M (1 - rho)/(1 + rho)."""
    rng = np.random.default_rng(2)
    M = 200_000
    e = rng.normal(size=M)
    x = np.empty(M)
    x[0] = e[0]
    for t in range(1, M):
        x[t] = rho * x[t - 1] + e[t]
    g = oracle.geyer_ims(x)
    want = M * (1 - rho) / (1 + rho)
    assert abs(g["ess"] / want - 1) < 0.08
    assert abs(g["se"] - np.sqrt(g["var"] / g["ess"])) < 1e-12
    assert abs(g["var"] - 1 / (1 - rho ** 2)) < 0.05 / (1 - rho ** 2)


def test_geyer_takes_the_initial_monotone_sequence():
    """x_t = cos(0.8 pi t): gamma(k) -> cos(0.8 pi k) / 2, so the pair sums are
    Gamma_0 = (1 + cos 0.8pi)/2, Gamma_1 = (cos 1.6pi + cos 2.4pi)/2 (larger),
    Gamma_2 = (cos 3.2pi + 1)/2, and Gamma_3 = (cos 4.8pi + cos 5.6pi)/2 < 0 ends the
    sequence.  The initial positive sequence sums Gamma_0..2 as they are (sigma^2 =
    gamma(0), effective length M); the initial monotone sequence caps Gamma_1 and
    Gamma_2 at Gamma_0, which gives sigma^2 = -1/2 + 6 Gamma_0 and an effective
    length of about 6.85 M.  Geyer (1992) as read for Sec. 2.3: the monotone one."""
    M = 10_000  # a whole number of periods (5 samples = 2 periods): the mean is 0
    x = np.cos(0.8 * np.pi * np.arange(M))
    g = oracle.geyer_ims(x)
    g0 = 0.5 * (1 + np.cos(0.8 * np.pi))
    want = M * 0.5 / (-0.5 + 6 * g0)
    assert abs(g["ess"] / want - 1) < 0.01
    assert g["ess"] > 6 * M  # the initial positive sequence would give about M


def test_trace_series_mean_is_the_diagonal_trace():
    """The realised per-cycle trace values average to sum_i q_i diag_i (Eq. tr)."""
    csr = _small_random(18, 9, complex_=True)
    q = np.random.default_rng(0).uniform(0, 1, 18)
    series = []
    st, dacc, _ = oracle.run(csr, 16, seed=3, ncycles=40, acc_from=10, q=q, series_out=series)
    st, dacc2, _ = oracle.run(csr, 16, seed=3, cycle0=40, ncycles=15, acc_from=10, state=st, q=q,
                              series_out=series)
    assert len(series) == 45
    tr = ((dacc.sum(0) + dacc2.sum(0)) * q).sum().real / (16 * 45)
    assert abs(np.mean(series) - tr) < 1e-12 * abs(tr)
