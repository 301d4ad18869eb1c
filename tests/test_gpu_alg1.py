"""Algorithm 1 on the GPU: the coupling burn-in (steps 1-5, Eq. 12), the
realised trace series and its Monte Carlo error by Geyer's effective length
(Sec. 2.3), and the stop rule (relative SE below tol, Sec. 3.1)."""
import numpy as np
import pytest

import oracle
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def gs_max_sequence(a, cycles):
    """max_i |d_i| after each noise-free Gauss-Seidel sweep on a d = 0 from d = (1..n)."""
    n = a.shape[0]
    d = np.arange(1, n + 1).astype(np.complex128)
    out = []
    for _ in range(cycles):
        for i in range(n):
            d[i] = -(a[i, :i] @ d[:i] + a[i, i + 1:] @ d[i + 1:]) / a[i, i]
        out.append(np.abs(d).max())
    return np.array(out)


@pytest.mark.parametrize("kind", ["real", "complex", "pedigree"])
def test_coupled_burnin_length(kind):
    if kind == "real":
        csr = wl.random_dominant(200, 4, 1.3, 3)
    elif kind == "complex":
        csr = wl.u1_lattice((9, 7), 0.2, 0.15, seed=2)
    else:
        csr = wl.pedigree(400, 1.2, 5)
    a = csr.to_dense().astype(np.complex128)
    mz = gs_max_sequence(a, 60)
    mw = gs_max_sequence(a.conj().T, 60)
    m = np.maximum(mz, mw)
    # a tolerance half-way (geometrically) between two consecutive maxima near 5e-5,
    # so FP32 rounding cannot move the crossing
    k = int(np.argmax(m < 5e-5))
    tol = float(np.sqrt(m[k] * m[k - 1]))
    h = mcinv.create_from_csr(csr, K=32, seed=1, acc=mcinv.MCINV_ACC_FP32_SIMT)
    p = mcinv.mcinv_burnin_coupled(h, tol, 1000)
    assert p == k + 1
    p_orc, _, _ = oracle.coupling_burnin(csr, seed=1, tol=tol)
    assert p_orc == p
    # the chains ran p burn-in cycles, exactly as a plain burn-in of p cycles
    z, w, cyc = mcinv.mcinv_get_state(h)
    h2 = mcinv.create_from_csr(csr, K=32, seed=1, acc=mcinv.MCINV_ACC_FP32_SIMT)
    mcinv.mcinv_burnin(h2, p)
    z2, w2, _ = mcinv.mcinv_get_state(h2)
    assert cyc == p and np.array_equal(z, z2) and np.array_equal(w, w2)


def test_coupled_burnin_reports_divergence():
    csr = wl.csr_from_coo(2, [0, 0, 1, 1], [0, 1, 0, 1], np.array([1.0, 3.0, 4.0, 1.0]))
    h = mcinv.create_from_csr(csr, K=4, acc=mcinv.MCINV_ACC_FP32_SIMT)
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_burnin_coupled(h, 1e-6, 50)
    assert e.value.status == 3


@pytest.mark.parametrize("complex_", [False, True])
def test_trace_series_matches_oracle(complex_):
    csr = wl.u1_lattice((8, 10), 0.12, 0.08, seed=4) if complex_ else wl.random_dominant(300, 4, 1.5, 8)
    q = wl.q_diag(csr.n, 2)
    K, burn, samp = 64, 5, 30
    h = mcinv.create_from_csr(csr, K=K, seed=6, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=8)
    mcinv.mcinv_set_trace_weights(h, q)
    mcinv.mcinv_burnin(h, burn)
    mcinv.mcinv_sample(h, samp)
    s_gpu = mcinv.mcinv_trace_series(h)
    s_orc = []
    oracle.run(csr, K, seed=6, ncycles=burn + samp, acc_from=burn, q=q, series_out=s_orc)
    s_orc = np.array(s_orc)
    assert len(s_gpu) == samp
    assert np.abs(s_gpu - s_orc).max() <= 1e-4 * np.abs(s_orc).max()
    g = mcinv.mcinv_trace_mc_error(h)
    g_orc = oracle.geyer_ims(s_gpu)  # the oracle's estimator on the GPU's own series
    for key in ("mean", "var", "ess", "se"):
        assert abs(g[key] - g_orc[key]) <= 1e-9 * abs(g_orc[key]), key


def test_stop_rule_reaches_the_relative_error():
    csr = wl.random_dominant(500, 4, 1.5, 12)
    q = np.ones(csr.n)
    h = mcinv.create_from_csr(csr, K=256, seed=2, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=10)
    mcinv.mcinv_set_trace_weights(h, q)
    mcinv.mcinv_burnin_coupled(h, 5e-5, 1000)
    used = mcinv.mcinv_sample_until(h, 2e-4, 100, 100_000)
    g = mcinv.mcinv_trace_mc_error(h)
    assert g["se"] < 2e-4 * abs(g["mean"]) and used % 100 == 0
    # one check earlier the rule was not met yet (unless the first check already met it)
    assert used >= 100
    tr, tse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_TRACE, q_diag=q)
    assert abs(tr - g["mean"]) <= 1e-9 * abs(tr)
    truth = np.trace(np.linalg.inv(csr.to_dense()))
    assert abs(tr - truth) < 5 * g["se"]
