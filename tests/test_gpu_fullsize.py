"""Parity at the workloads' full sizes, in the launch configuration the benchmark
times (autotuned slice shape, both sweep orders): the oracle follows a few sampled
chains (it can run any chain range on its own), and the GPU state of those chains
must match it after a few cycles.  Bar: 1e-4 relative, as for the small cases."""
import numpy as np
import pytest

import oracle
from _greedy import greedy_order, permuted
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-4

CASES = {
    "pedigree50k": (lambda: wl.WORKLOADS["pedigree50k"].build(), 1024, [0, 517, 1020]),
    "lattice2d128": (lambda: wl.WORKLOADS["lattice2d128"].build(), 4096, [0, 2049, 4094]),
    "lattice4d16": (lambda: wl.WORKLOADS["lattice4d16"].build(), 8192, [0, 4097]),
    "dirac18": (lambda: wl.wilson_dirac((18, 18, 18, 18), 0.1), 1024, [0, 1022]),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("order", ["natural", "colour"])
@pytest.mark.parametrize("name", list(CASES))
def test_sampled_chains_match_the_oracle(name, order):
    make, K, chains = CASES[name]
    c = make()
    flags = mcinv.MCINV_F_AUTOTUNE | (mcinv.MCINV_F_COLOR_ORDER if order == "colour" else 0)
    cycles = 3
    h = mcinv.create_from_csr(c, K=K, seed=11, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=cycles, flags=flags)
    mcinv.mcinv_burnin(h, cycles)
    if order == "colour":
        o, _ = greedy_order(c)
        cref = permuted(c, o)
    else:
        o, cref = None, c
    for c0 in chains:
        nch = min(2, K - c0)
        z, w, cyc = mcinv.mcinv_get_state(h, c0, nch)
        assert cyc == cycles
        st, _, _ = oracle.run(cref, nch, seed=11, chain0=c0, ncycles=cycles, diag=False)
        zr, wr = (z[o], w[o]) if o is not None else (z, w)
        assert _rel(zr, st.z) <= TOL and _rel(wr, st.w) <= TOL, (name, order, c0, _rel(zr, st.z), _rel(wr, st.w))
    mcinv.mcinv_destroy(h)


def _bench_handle(name, c, K):
    """The handle as the benchmark creates it for this workload: autotuned kernel,
    colour order, and the workload's estimates accumulated while sampling."""
    flags = mcinv.MCINV_F_AUTOTUNE | mcinv.MCINV_F_COLOR_ORDER
    if name == "pedigree50k":  # diagonal + C^-1[:, 0:512] on the tensor cores
        return mcinv.create_from_csr(c, K=K, seed=11, acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=8, flags=flags,
                                     block_rows=np.arange(c.n), block_cols=np.arange(512))
    if name == "lattice4d16":  # C^-1[0:4096, 0:4096] on the tensor cores
        R = np.arange(4096)
        return mcinv.create_from_csr(c, K=K, seed=11, acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=8, flags=flags,
                                     block_rows=R, block_cols=R)
    # lattice2d128 and the Wilson-Dirac matrix: diagonal and trace
    h = mcinv.create_from_csr(c, K=K, seed=11, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=8, flags=flags)
    mcinv.mcinv_set_trace_weights(h, wl.q_diag(c.n, 0))
    return h


@pytest.mark.parametrize("name", list(CASES))
def test_sampled_chains_follow_the_oracle_for_100_cycles(name):
    """Same-draw parity at full size over 100 cycles (20 burn-in, then 80 sampling
    cycles with the estimates accumulated) in the benchmark's configuration, for
    two chains in the middle of the chain range, checked after cycles 20 and 100."""
    make, K, _ = CASES[name]
    c = make()
    h = _bench_handle(name, c, K)
    o, _ = greedy_order(c)
    cref = permuted(c, o)
    c0, nch = K // 2 + 1, 2
    st = None
    for done, todo in ((0, 20), (20, 80)):
        if done == 0:
            mcinv.mcinv_burnin(h, todo)
        else:
            mcinv.mcinv_sample(h, todo)
        z, w, cyc = mcinv.mcinv_get_state(h, c0, nch)
        assert cyc == done + todo
        st, _, _ = oracle.run(cref, nch, seed=11, chain0=c0, cycle0=done, ncycles=todo, diag=False, state=st)
        ez, ew = _rel(z[o], st.z), _rel(w[o], st.w)
        assert ez <= TOL and ew <= TOL, (name, cyc, ez, ew)
    mcinv.mcinv_destroy(h)
