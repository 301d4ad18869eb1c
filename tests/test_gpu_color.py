"""The colour sweep order on the GPU (MCINV_F_COLOR_ORDER): the handle samples
C' = P C P^T (Sec. 4, reordering C), so its chains must follow the oracle's
same-draw trajectory on C' (built here from the order's definition), and its
estimates, mapped back to the rows of C, must estimate C^-1."""
import numpy as np
import pytest

import oracle
from _greedy import greedy_order, permuted
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-4
COLOR = mcinv.MCINV_F_COLOR_ORDER


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("make,K,shape", [
    (lambda: wl.pedigree(3000, 1.2, 1), 40, {}),
    (lambda: wl.random_dominant(256, 4, 1.5, 0), 128, {"chains_per_cta": 32, "threads_per_cta": 256, "ctas_per_slice": 4}),
    (lambda: wl.u1_lattice((16, 12), 0.12, 0.08, seed=2), 24, {}),
    (lambda: wl.wilson_dirac((3, 3, 3, 4), 0.1), 48, {"chains_per_cta": 16, "threads_per_cta": 128}),
])
def test_trajectory_is_the_oracle_on_the_permuted_matrix(make, K, shape):
    c = make()
    order, _ = greedy_order(c)
    cp = permuted(c, order)
    h = mcinv.create_from_csr(c, K=K, seed=3, acc=mcinv.MCINV_ACC_FP32_SIMT, flags=COLOR, **shape)
    info = mcinv.mcinv_info(h)
    assert info["levels"] <= int(np.max(greedy_order(c)[1])) + 1
    st, done = None, 0
    for cyc in (1, 10, 60):
        mcinv.mcinv_burnin(h, cyc - done)
        st, _, _ = oracle.run(cp, K, seed=3, cycle0=done, ncycles=cyc - done, state=st)
        done = cyc
        z, w, _ = mcinv.mcinv_get_state(h)
        # the library returns rows of C: row order[k] of z is row k of the oracle's C' state
        assert _rel(z[order], st.z) <= TOL and _rel(w[order], st.w) <= TOL, cyc
    mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("complex_", [False, True])
def test_estimates_in_the_rows_of_c(complex_):
    c = wl.u1_lattice((10, 12), 0.2, 0.15, seed=4) if complex_ else wl.random_dominant(240, 4, 1.4, 6)
    inv = np.linalg.inv(c.to_dense())
    R = np.arange(0, c.n, 3)
    S = np.array([5, 0, 17, 101, 64])
    h = mcinv.create_from_csr(c, K=256, seed=8, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=10, flags=COLOR,
                              block_rows=R, block_cols=S)
    q = wl.q_diag(c.n, 5)
    mcinv.mcinv_set_trace_weights(h, q)
    mcinv.mcinv_burnin(h, 60)
    mcinv.mcinv_sample(h, 400)
    d, dse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_DIAG)
    b, bse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
    tr, tse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_TRACE, q_diag=q)
    g = mcinv.mcinv_trace_mc_error(h)
    mcinv.mcinv_destroy(h)
    re = (lambda x: x.real) if complex_ else (lambda x: x)
    zd = np.abs(re(d) - re(np.diag(inv))) / re(dse)
    zb = np.abs(re(b) - re(inv[np.ix_(R, S)])) / re(bse)
    for zz in (zd, zb.ravel()):
        assert (zz > 3.5).mean() < 0.02 and 0.7 < np.sqrt(np.mean(zz ** 2)) < 1.35
    exact_tr = (q * np.diag(inv)).sum()
    assert abs(re(tr) - re(exact_tr)) < 4 * re(tse)
    assert abs(g["mean"] - re(exact_tr)) < 4 * g["se"]


def test_resume_is_bit_exact_in_colour_order():
    c = wl.pedigree(1500, 1.2, 2)
    h = mcinv.create_from_csr(c, K=64, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, flags=COLOR)
    mcinv.mcinv_burnin(h, 7)
    z, w, cyc = mcinv.mcinv_get_state(h)
    mcinv.mcinv_burnin(h, 5)
    z1, w1, _ = mcinv.mcinv_get_state(h)
    h2 = mcinv.create_from_csr(c, K=64, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, flags=COLOR)
    mcinv.mcinv_set_state(h2, z, w, cyc)
    mcinv.mcinv_burnin(h2, 5)
    z2, w2, _ = mcinv.mcinv_get_state(h2)
    assert np.array_equal(z1, z2) and np.array_equal(w1, w2)
    mcinv.mcinv_destroy(h)
    mcinv.mcinv_destroy(h2)


def test_tensor_core_block_in_colour_order():
    c = wl.pedigree(2000, 1.2, 3)
    inv = np.linalg.inv(c.to_dense())
    S = np.arange(0, 300)
    h = mcinv.create_from_csr(c, K=512, seed=2, acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=8, flags=COLOR,
                              block_rows=np.arange(c.n), block_cols=S)
    mcinv.mcinv_burnin(h, 40)
    mcinv.mcinv_sample(h, 160)
    b, bse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
    mcinv.mcinv_destroy(h)
    zb = np.abs(b - inv[:, S]) / np.maximum(bse, 1e-12)
    assert (zb > 4).mean() < 0.02 and np.sqrt(np.mean(zb ** 2)) < 1.4
