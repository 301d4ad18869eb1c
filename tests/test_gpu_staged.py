"""The staged sweep (MCINV_F_STAGED): a producer warp stages the gathers in shared
memory with bulk copies on mbarriers, consumer warps do the arithmetic of the
register kernel in the same order.  So for every shape its chains, diagonal and
block must equal the register kernel's bit for bit, and follow the oracle."""
import numpy as np
import pytest

import oracle
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ST = mcinv.MCINV_F_STAGED
CO = mcinv.MCINV_F_COLOR_ORDER


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def _pair(c, K, W, Q, flags=0, cycles=(1, 7, 25), **kw):
    hs = mcinv.create_from_csr(c, K=K, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, chains_per_cta=W,
                               ctas_per_slice=Q, flags=flags | ST, **kw)
    hr = mcinv.create_from_csr(c, K=K, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, chains_per_cta=W,
                               ctas_per_slice=Q, threads_per_cta=256, flags=flags, **kw)
    done = 0
    for cyc in cycles:
        for h in (hs, hr):
            mcinv.mcinv_burnin(h, cyc - done)
        done = cyc
        zs, ws, _ = mcinv.mcinv_get_state(hs)
        zr, wr, _ = mcinv.mcinv_get_state(hr)
        assert np.array_equal(zs, zr) and np.array_equal(ws, wr), cyc
    return hs, hr


@pytest.mark.parametrize("W,Q", [(16, 1), (32, 1), (32, 2), (32, 4), (16, 8)])
def test_staged_equals_register_kernel(W, Q):
    c = wl.pedigree(6000, 1.2, 3)  # long rows (split items) and 60-odd levels
    hs, hr = _pair(c, 128, W, Q)
    for h in (hs, hr):
        mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("flags", [0, CO])
def test_staged_equals_register_kernel_with_estimates(flags):
    c = wl.random_dominant(700, 4, 1.5, 9)
    hs, hr = _pair(c, 256, 32, 2, flags=flags, cycles=(5,), batch_cycles=4)
    for h in (hs, hr):
        mcinv.mcinv_sample(h, 20)
    ds, _ = mcinv.mcinv_estimate(hs, mcinv.MCINV_EST_DIAG)
    dr, _ = mcinv.mcinv_estimate(hr, mcinv.MCINV_EST_DIAG)
    assert np.array_equal(ds, dr)
    for h in (hs, hr):
        mcinv.mcinv_destroy(h)


def test_staged_trace_series_and_tensor_core_block():
    c = wl.pedigree(3000, 1.2, 7)
    q = wl.q_diag(c.n, 1)
    hs = mcinv.create_from_csr(c, K=512, seed=2, acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=8, chains_per_cta=32,
                               ctas_per_slice=2, flags=ST, block_rows=np.arange(c.n), block_cols=np.arange(256))
    hr = mcinv.create_from_csr(c, K=512, seed=2, acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=8, chains_per_cta=32,
                               ctas_per_slice=2, threads_per_cta=256,
                               block_rows=np.arange(c.n), block_cols=np.arange(256))
    for h in (hs, hr):
        mcinv.mcinv_set_trace_weights(h, q)
        mcinv.mcinv_burnin(h, 10)
        mcinv.mcinv_sample(h, 32)
    bs, _ = mcinv.mcinv_estimate(hs, mcinv.MCINV_EST_BLOCK)
    br, _ = mcinv.mcinv_estimate(hr, mcinv.MCINV_EST_BLOCK)
    assert np.array_equal(bs, br)  # same shadows, same contraction
    ss = mcinv.mcinv_trace_series(hs)
    sr = mcinv.mcinv_trace_series(hr)
    assert len(ss) == 32 and np.abs(ss - sr).max() <= 1e-5 * np.abs(sr).max()  # FP32 partials, other order
    for h in (hs, hr):
        mcinv.mcinv_destroy(h)


def test_staged_follows_the_oracle():
    c = wl.pedigree(2000, 1.2, 11)
    h = mcinv.create_from_csr(c, K=64, seed=8, acc=mcinv.MCINV_ACC_FP32_SIMT, chains_per_cta=16, ctas_per_slice=2,
                              flags=ST)
    mcinv.mcinv_burnin(h, 30)
    z, w, _ = mcinv.mcinv_get_state(h)
    st, _, _ = oracle.run(c, 64, seed=8, ncycles=30)
    assert np.abs(z - st.z.real).max() <= 1e-4 * np.abs(st.z).max()
    assert np.abs(w - st.w.real).max() <= 1e-4 * np.abs(st.w).max()
    mcinv.mcinv_destroy(h)


def test_staged_rejections():
    c = wl.random_dominant(100, 4, 1.5, 1)
    with pytest.raises(mcinv.McinvError) as e:  # 64-chain slices: split rows would span two rounds
        mcinv.create_from_csr(c, K=128, chains_per_cta=64, flags=ST)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    with pytest.raises(mcinv.McinvError) as e:  # K not a multiple of the 32-chain slice
        mcinv.create_from_csr(c, K=48, chains_per_cta=32, flags=ST)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    z = wl.u1_lattice((8, 8), 0.1, 0.1, seed=1)
    with pytest.raises(mcinv.McinvError) as e:  # complex
        mcinv.create_from_csr(z, K=64, chains_per_cta=16, flags=ST)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
