"""GPU parity of the coupled sweep and its estimates against the FP64 oracle.

Same-draw trajectories: both sides draw phi from Philox4x32-10 keyed by
(seed, chain, cycle, row, matrix), so after k cycles the GPU state must equal
the oracle's up to FP32 rounding.  Bar: max_{i,c} |z_gpu - z_orc| /
max_{i,c} |z_orc| <= 1e-4 over 100 cycles (and the same for w).
"""
import numpy as np
import pytest

import oracle
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def rel_err(gpu, orc):
    return np.abs(gpu - orc).max() / max(np.abs(orc).max(), 1e-30)


def run_pair(csr, K, cycles, seed=3, matrix_id=0, chain_base=0, **kw):
    h = mcinv.create_from_csr(csr, K=K, seed=seed, matrix_id=matrix_id, chain_base=chain_base,
                              acc=mcinv.MCINV_ACC_FP32_SIMT, **kw)
    st = None
    done = 0
    out = []
    for c in cycles:
        mcinv.mcinv_burnin(h, c - done)
        st, _, _ = oracle.run(csr, K, seed=seed, matrix=matrix_id, chain0=chain_base, cycle0=done,
                              ncycles=c - done, state=st)
        done = c
        z, w, cyc = mcinv.mcinv_get_state(h)
        assert cyc == c
        out.append((rel_err(z, st.z), rel_err(w, st.w)))
    return h, st, out


def _assert_close(errs):
    for ez, ew in errs:
        assert ez <= TOL and ew <= TOL, errs


# -- trajectories on the workload families, small sizes spanning several tiles -----------------

def test_trajectory_random256():
    csr = wl.random_dominant(256, 4, 1.5, 0)
    _, _, errs = run_pair(csr, 128, [1, 10, 100])
    _assert_close(errs)


def test_trajectory_pedigree_small():
    csr = wl.pedigree(3000, 1.2, 1)
    _, _, errs = run_pair(csr, 40, [1, 10, 100])
    _assert_close(errs)


def test_trajectory_lattice2d_complex():
    csr = wl.u1_lattice((16, 12), 0.12, 0.08, seed=2)
    _, _, errs = run_pair(csr, 24, [1, 10, 100])
    _assert_close(errs)


def test_trajectory_lattice4d_complex():
    csr = wl.u1_lattice((4, 3, 4, 3), 0.06, 0.04, seed=5)
    _, _, errs = run_pair(csr, 33, [1, 30])
    _assert_close(errs)


@pytest.mark.parametrize("W", [1, 2, 4, 8, 16, 32, 64, 128])
@pytest.mark.parametrize("threads", [32, 256, 512])
@pytest.mark.parametrize("K", [45, 200])
def test_trajectory_every_slice_shape(W, threads, K):
    """Every chain-slice width and block size gives the same sweep: K = 45 runs one
    chain per lane with a ragged last slice, K = 200 the vector path (4 chains per
    lane) with a ragged last slice."""
    csr = wl.random_dominant(300, 5, 1.3, 7)
    if K % 4 and W > 32:  # one chain per lane: at most 32 lanes per row
        with pytest.raises(mcinv.McinvError) as e:
            mcinv.create_from_csr(csr, K=K, chains_per_cta=W, acc=mcinv.MCINV_ACC_FP32_SIMT)
        assert e.value.status == 1
        return
    _, _, errs = run_pair(csr, K, [3], chains_per_cta=W, threads_per_cta=threads)
    _assert_close(errs)


@pytest.mark.parametrize("W", [1, 2, 8, 32, 64])
@pytest.mark.parametrize("K", [33, 66])
def test_trajectory_complex_slice_shapes(W, K):
    """Complex sweep: one chain per lane (K = 33) and two per lane (K = 66)."""
    csr = wl.u1_lattice((7, 9), 0.12, 0.08, seed=8)
    if K % 2 and W > 32:
        return
    _, _, errs = run_pair(csr, K, [4], chains_per_cta=W, threads_per_cta=128)
    _assert_close(errs)


@pytest.mark.parametrize("Q", [2, 3, 8, 16])
@pytest.mark.parametrize("W,threads", [(64, 512), (32, 128), (128, 256)])
def test_trajectory_cluster_slices(Q, W, threads):
    """A thread-block cluster of Q CTAs per chain slice (rows of each level split
    across the cluster, cluster barrier between levels) gives the same sweep."""
    csr = wl.pedigree(3000, 1.2, 3)
    _, _, errs = run_pair(csr, 256, [2, 12], chains_per_cta=W, threads_per_cta=threads, ctas_per_slice=Q)
    _assert_close(errs)


def test_trajectory_cluster_complex():
    csr = wl.u1_lattice((6, 5, 4, 3), 0.06, 0.04, seed=9)
    _, _, errs = run_pair(csr, 128, [3], chains_per_cta=64, threads_per_cta=256, ctas_per_slice=4)
    _assert_close(errs)


@pytest.mark.parametrize("complex_", [False, True])
def test_autotuned_shape_keeps_the_trajectory(complex_):
    """MCINV_F_AUTOTUNE times candidate shapes from the zero state, then restores it:
    the tuned handle starts at cycle 0 and follows the oracle."""
    csr = wl.u1_lattice((12, 10), 0.12, 0.08, seed=1) if complex_ else wl.pedigree(4000, 1.2, 2)
    h, st, errs = run_pair(csr, 64, [1, 7], flags=mcinv.MCINV_F_AUTOTUNE)
    _assert_close(errs)
    info = mcinv.mcinv_info(h)
    assert info["kernel_launches"] > 4 and info["cycle"] == 7


def test_default_shape_uses_clusters_for_few_slices():
    csr = wl.pedigree(2000, 1.2, 4)
    h = mcinv.create_from_csr(csr, K=1024, acc=mcinv.MCINV_ACC_FP32_SIMT)
    info = mcinv.mcinv_info(h)
    assert info["slices"] * info["ctas_per_slice"] >= 128
    assert info["chains_per_lane"] == 4


def test_trajectory_chain_base_and_matrix_id():
    csr = wl.random_dominant(100, 3, 1.5, 2)
    _, _, errs = run_pair(csr, 20, [5], seed=2 ** 40 + 17, matrix_id=9, chain_base=1000)
    _assert_close(errs)


# -- special cases ----------------------------------------------------------------------------

def test_single_row_and_single_chain():
    csr = wl.CSR(1, np.array([0, 1]), np.array([0], dtype=np.int32), np.array([2.5]))
    _, _, errs = run_pair(csr, 1, [1, 4])
    _assert_close(errs)


@pytest.mark.parametrize("complex_", [False, True])
def test_diagonal_matrix_noise_exact(complex_):
    """Diagonal C: z_i = phi_i/sqrt(c_ii) exactly -> checks every noise bit, and each
    sample z_i conj(w_i) = 1/c_ii."""
    n, K = 777, 70
    rng = np.random.default_rng(0)
    d = rng.uniform(0.5, 2.0, n) * rng.choice([-1.0, 1.0], n)
    if complex_:
        d = d * np.exp(1j * rng.uniform(-1, 1, n))
    csr = wl.CSR(n, np.arange(n + 1), np.arange(n, dtype=np.int32), d)
    h = mcinv.create_from_csr(csr, K=K, seed=11, acc=mcinv.MCINV_ACC_FP32_SIMT)
    mcinv.mcinv_sample(h, 3)
    z, w, _ = mcinv.mcinv_get_state(h)
    st, _, _ = oracle.run(csr, K, seed=11, ncycles=3)
    assert rel_err(z, st.z) < 1e-6 and rel_err(w, st.w) < 1e-6
    m, _ = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_DIAG)
    assert np.allclose(m, 1 / d, rtol=1e-6)


def test_hermitian_gives_w_equal_z():
    b = wl.random_dominant(200, 3, 1.0, 4).to_dense()
    h_ = b + b.T
    np.fill_diagonal(h_, np.abs(h_).sum(axis=1) + 1.0)
    csr = wl.csr_from_coo(200, *np.nonzero(h_), h_[np.nonzero(h_)])
    h = mcinv.create_from_csr(csr, K=32, seed=1, acc=mcinv.MCINV_ACC_FP32_SIMT)
    mcinv.mcinv_burnin(h, 20)
    z, w, _ = mcinv.mcinv_get_state(h)
    assert np.abs(z - w).max() <= 1e-5 * np.abs(z).max()


def test_divergence_is_reported():
    """C = [[1,a],[b,1]] with |ab| > 1: sp(T) > 1, the chains blow up (Sec. 2.2)."""
    csr = wl.csr_from_coo(2, [0, 0, 1, 1], [0, 1, 0, 1], np.array([1.0, 3.0, 4.0, 1.0]))
    h = mcinv.create_from_csr(csr, K=8, seed=1, acc=mcinv.MCINV_ACC_FP32_SIMT)
    mcinv.mcinv_burnin(h, 60)
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_sync(h)
    assert e.value.status == 3


def test_resume_is_bit_exact():
    csr = wl.random_dominant(500, 4, 1.5, 3)
    a = mcinv.create_from_csr(csr, K=64, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT)
    mcinv.mcinv_burnin(a, 20)
    za, wa, _ = mcinv.mcinv_get_state(a)
    b = mcinv.create_from_csr(csr, K=64, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT)
    mcinv.mcinv_burnin(b, 9)
    z9, w9, c9 = mcinv.mcinv_get_state(b)
    c = mcinv.create_from_csr(csr, K=64, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT)
    mcinv.mcinv_set_state(c, z9, w9, c9)
    mcinv.mcinv_burnin(c, 11)
    zc, wc, cc = mcinv.mcinv_get_state(c)
    assert cc == 20 and np.array_equal(za, zc) and np.array_equal(wa, wc)


# -- estimates against the oracle's accumulation of the same draws ---------------------------------

@pytest.mark.parametrize("complex_", [False, True])
def test_estimates_match_oracle_same_draws(complex_):
    if complex_:
        csr = wl.u1_lattice((10, 9), 0.12, 0.08, seed=3)
    else:
        csr = wl.random_dominant(90, 4, 1.5, 5)
    n, K, burn, samp = csr.n, 64, 7, 13
    R = np.arange(0, n, 3)
    S = np.arange(1, n, 4)
    h = mcinv.create_from_csr(csr, K=K, seed=8, acc=mcinv.MCINV_ACC_FP32_SIMT, chains_per_cta=4,
                              groups=16, batch_cycles=4, block_rows=R, block_cols=S)
    info = mcinv.mcinv_info(h)
    assert info["groups"] == 16
    mcinv.mcinv_burnin(h, burn)
    mcinv.mcinv_sample(h, samp)
    dm, dse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_DIAG)
    bm, bse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
    q = wl.q_diag(n, 1)
    tm, tse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_TRACE, q_diag=q)
    st, dacc, bacc = oracle.run(csr, K, seed=8, ncycles=burn + samp, acc_from=burn, cpg=4, R=R, S=S)
    om, ose = oracle.group_estimate(dacc, np.full(16, 4), samp)
    assert rel_err(dm, om) < TOL
    assert rel_err(dse, ose) < 1e-3
    ob = bacc.sum(0) / (K * samp)
    assert rel_err(bm, ob) < TOL
    tg = (dacc * q[None, :]).sum(axis=1)
    otm, otse = oracle.group_estimate(tg, np.full(16, 4), samp)
    assert abs(tm - otm) <= TOL * np.abs(om * q).sum()
    assert abs(tse.real - otse.real) <= 1e-3 * abs(otse.real)


def test_block_standard_error_is_batch_means():
    """Block SE = SE of the per-batch means (Sec. 2.3), recomputed from the oracle's
    per-batch sums of the same draws."""
    csr = wl.random_dominant(60, 3, 1.5, 9)
    K, B, nb = 32, 5, 6
    R = np.arange(10)
    h = mcinv.create_from_csr(csr, K=K, seed=4, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=B,
                              block_rows=R, block_cols=R)
    mcinv.mcinv_sample(h, B * nb)
    bm, bse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
    st = None
    means = []
    for b in range(nb):
        st, _, bacc = oracle.run(csr, K, seed=4, cycle0=b * B, ncycles=B, acc_from=b * B, state=st,
                                 R=R, S=R, diag=False)
        means.append(bacc.sum(0).real / (K * B))
    means = np.array(means)
    want_se = means.std(axis=0, ddof=1) / np.sqrt(nb)
    assert rel_err(bm, means.mean(0)) < TOL
    assert np.abs(bse - want_se).max() <= 1e-3 * want_se.max()


# -- statistics: config "random256" end to end against the dense inverse ---------------------------

def test_random256_full_inverse_within_3se_of_lu():
    csr = wl.random_dominant(256, 4, 1.5, 0)
    n = 256
    R = np.arange(n)
    h = mcinv.create_from_csr(csr, K=128, seed=0, acc=mcinv.MCINV_ACC_FP32_SIMT, block_rows=R,
                              block_cols=R, batch_cycles=50)
    mcinv.mcinv_burnin(h, 200)
    mcinv.mcinv_sample(h, 2000)
    m, se = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
    truth = np.linalg.inv(csr.to_dense())
    zs = (m - truth) / se
    assert np.mean(np.abs(zs) > 3) < 0.01
    assert 0.8 < np.sqrt(np.mean(zs ** 2)) < 1.25
    dm, dse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_DIAG)
    zd = (dm - np.diag(truth)) / dse
    assert np.mean(np.abs(zd) > 3) < 0.03


# -- full-size workloads, sampled chains recomputed by the oracle one by one -------------------------

@pytest.mark.parametrize("name,cycles", [("pedigree50k", 2), ("lattice2d128", 2), ("lattice4d16", 1)])
def test_full_size_sampled_chains(name, cycles):
    w = wl.WORKLOADS[name]
    csr = w.build()
    h = mcinv.create_from_csr(csr, K=w.K, seed=0, acc=mcinv.MCINV_ACC_FP32_SIMT)
    mcinv.mcinv_burnin(h, cycles)
    rng = np.random.default_rng(1)
    for c in sorted(rng.choice(w.K, size=3, replace=False)):
        z, wv, _ = mcinv.mcinv_get_state(h, int(c), 1)
        st, _, _ = oracle.run(csr, 1, seed=0, chain0=int(c), ncycles=cycles)
        assert rel_err(z, st.z) < TOL and rel_err(wv, st.w) < TOL
