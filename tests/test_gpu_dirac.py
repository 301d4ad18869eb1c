"""Example 2 on the GPU: the free Wilson-Dirac matrix (Sec. 3.2, Eq. explicit).

Same-draw trajectories against the FP64 oracle (14 nonzeros per row, so every row
runs two passes of the unrolled gather loop), the trace and diagonal estimates after
the coupling burn-in against the momentum-space closed form of L^-1, and the same at
the paper's 18^4 lattice (Table 3, case 1), where the oracle cannot follow: there the
check is the exact trace within the run's own MC error.
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


def _rel(gpu, orc):
    return np.abs(gpu - orc).max() / max(np.abs(orc).max(), 1e-30)


@pytest.mark.parametrize("shape", [{}, {"chains_per_cta": 32, "threads_per_cta": 256, "ctas_per_slice": 4},
                                   {"chains_per_cta": 8, "threads_per_cta": 128}])
def test_trajectory_dirac(shape):
    csr = wl.wilson_dirac((3, 3, 3, 4), 0.1)
    K = 48
    h = mcinv.create_from_csr(csr, K=K, seed=4, acc=mcinv.MCINV_ACC_FP32_SIMT, **shape)
    st, done = None, 0
    for c in (1, 10, 60):
        mcinv.mcinv_burnin(h, c - done)
        st, _, _ = oracle.run(csr, K, seed=4, cycle0=done, ncycles=c - done, state=st)
        done = c
        z, w, cyc = mcinv.mcinv_get_state(h)
        assert cyc == c
        assert _rel(z, st.z) <= TOL and _rel(w, st.w) <= TOL, (c, _rel(z, st.z), _rel(w, st.w))
    mcinv.mcinv_destroy(h)


def test_trace_and_diagonal_match_the_closed_form():
    dims = (6, 6, 6, 6)
    csr = wl.wilson_dirac(dims, 0.1)
    V = int(np.prod(dims))
    exact_blk = wl.wilson_dirac_propagator(dims, 0.1)
    exact_tr = wl.wilson_dirac_inverse_trace(dims, 0.1).real
    h = mcinv.create_from_csr(csr, K=256, seed=9, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=10)
    q = np.ones(csr.n)
    mcinv.mcinv_set_trace_weights(h, q)
    p = mcinv.mcinv_burnin_coupled(h, 1e-5, 500)
    assert 10 < p < 100
    mcinv.mcinv_sample(h, 300)
    tr, tse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_TRACE, q_diag=q)
    g = mcinv.mcinv_trace_mc_error(h)
    assert abs(tr.real - exact_tr) < 4 * g["se"] and g["se"] < 2e-4 * exact_tr
    assert abs(tr.real - exact_tr) < 4 * tse.real and abs(tr.imag) < 4 * tse.imag
    d, dse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_DIAG)
    want = np.repeat(np.diag(exact_blk), V)  # spinor index slowest
    z = np.abs(d.real - want.real) / dse.real
    assert (z > 3).mean() < 0.01 and 0.8 < np.sqrt(np.mean(z ** 2)) < 1.25
    mcinv.mcinv_destroy(h)


def test_paper_lattice_18_trace_within_its_error():
    """Table 3 case 1 (n = 419,904): coupling burn-in at tol 1e-5, then the trace at
    relative MC error below 1e-5, checked every 100 cycles (the rule of Tables 4, 5)."""
    csr = wl.wilson_dirac((18, 18, 18, 18), 0.1)
    exact = wl.wilson_dirac_inverse_trace((18,) * 4, 0.1).real
    h = mcinv.create_from_csr(csr, K=256, seed=1, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=10)
    q = np.ones(csr.n)
    mcinv.mcinv_set_trace_weights(h, q)
    p = mcinv.mcinv_burnin_coupled(h, 1e-5, 500)
    assert 20 < p < 80
    used = mcinv.mcinv_sample_until(h, 1e-5, 100, 5000)
    g = mcinv.mcinv_trace_mc_error(h)
    assert g["se"] < 1e-5 * abs(g["mean"]) and used % 100 == 0
    assert abs(g["mean"] - exact) < 4 * g["se"]
    mcinv.mcinv_destroy(h)
