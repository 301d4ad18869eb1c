"""The wavefront sweep (sweep_wave.cu): a CTA owns a slice of the chains for whole
cycles and walks the two colours of a lattice in the colour order as a wavefront
(red chunk t from the black chunks around it, then black chunk t - B from the new
red chunks), with no grid barrier.  Its arithmetic is every other kernel's, so the
chains must equal the chain-sliced kernel's bit for bit, over slice widths of 16,
8 and 4 vectors, bands of one, two and eight chunks, complex and real matrices, ragged
last slices and noise words, and with the estimates (diagonal partials, trace
series, BF16 shadows of a block) accumulated while sampling; and they must follow
the oracle's same-draw trajectories for 100 cycles."""
import numpy as np
import pytest

import oracle
from _greedy import greedy_order, permuted
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
WAVE = mcinv.MCINV_F_GRID | mcinv.MCINV_F_GRID_BULK | mcinv.MCINV_F_GRID_WAVE
CO = mcinv.MCINV_F_COLOR_ORDER


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def _real(c):
    """The same pattern with the real parts (a real non-symmetric, structurally symmetric C)."""
    return wl.CSR(c.n, c.row_ptr, c.col, np.ascontiguousarray(c.val.real))


def _slices(c, K, sv):
    V = 2 if np.iscomplexobj(c.val) else 4
    return (K // V + sv - 1) // sv


def _pair(c, K, sv, cycles=(1, 6, 20)):
    W = 64 if np.iscomplexobj(c.val) else 128
    ht = mcinv.create_from_csr(c, K=K, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=8, flags=WAVE | CO)
    hr = mcinv.create_from_csr(c, K=K, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=8, chains_per_cta=W,
                               ctas_per_slice=1, threads_per_cta=256, flags=CO)
    info = mcinv.mcinv_info(ht)
    assert info["sweep_kernel"] == 6 and info["threads_per_cta"] == 512
    assert info["grid_ctas"] == _slices(c, K, sv), info  # one CTA a chain slice of sv vectors
    done = 0
    for cyc in cycles:
        for h in (ht, hr):
            mcinv.mcinv_burnin(h, cyc - done)
        done = cyc
        zt, wt, _ = mcinv.mcinv_get_state(ht)
        zr, wr, _ = mcinv.mcinv_get_state(hr)
        assert np.array_equal(zt, zr) and np.array_equal(wt, wr), cyc
    for h in (ht, hr):
        mcinv.mcinv_destroy(h)


# (matrix, K, the slice width the form takes): 16-site half-rows in 32-position chunks
# (band 1) and 64-site half-rows (band 2); ragged last slices (K / V not a multiple of
# the width) and noise words (K not a multiple of 32)
CASES = [
    ("c16x16", lambda: wl.u1_lattice((16, 16), 0.12, 0.08, seed=2), 130, 4),
    ("c24x20", lambda: wl.u1_lattice((24, 20), 0.12, 0.08, seed=3), 520, 4),
    ("c32x32", lambda: wl.u1_lattice((32, 32), 0.12, 0.08, seed=4), 3100, 16),
    ("c128x16", lambda: wl.u1_lattice((128, 16), 0.12, 0.08, seed=5), 2000, 8),
    ("r32x32", lambda: _real(wl.u1_lattice((32, 32), 0.12, 0.08, seed=6)), 4000, 8),
    # 64 real chains a slice: two noise words, one for each of a lane's two vectors
    ("r32x32w", lambda: _real(wl.u1_lattice((32, 32), 0.12, 0.08, seed=14)), 6400, 16),
    ("r20x16", lambda: _real(wl.u1_lattice((20, 16), 0.12, 0.08, seed=7)), 132, 4),
    ("c8x8x8x8", lambda: wl.u1_lattice((8, 8, 8, 8), 0.06, 0.04, seed=8), 520, 4),  # band of 8 chunks
]


@pytest.mark.parametrize("name,make,K,sv", CASES, ids=[c[0] for c in CASES])
def test_wave_sweep_equals_chain_sliced_kernel(name, make, K, sv):
    _pair(make(), K, sv)


@pytest.mark.parametrize("make,K", [(lambda: wl.u1_lattice((16, 16), 0.12, 0.08, seed=6), 512),
                                    (lambda: wl.u1_lattice((32, 32), 0.12, 0.08, seed=9), 3200),
                                    # 64-site half-rows in 32-position chunks: band 2, slices of 16
                                    # (the shape of the 128 x 128 lattice at K = 4096)
                                    (lambda: wl.u1_lattice((128, 32), 0.12, 0.08, seed=13), 4096),
                                    (lambda: _real(wl.u1_lattice((16, 12), 0.12, 0.08, seed=7)), 512)])
def test_wave_estimates_equal_chain_sliced_kernel(make, K):
    c = make()
    q = wl.q_diag(c.n, 1)
    W = 64 if np.iscomplexobj(c.val) else 128
    kw = dict(acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=8, block_rows=np.arange(c.n), block_cols=np.arange(64))
    ht = mcinv.create_from_csr(c, K=K, seed=2, flags=WAVE | CO, **kw)
    hr = mcinv.create_from_csr(c, K=K, seed=2, chains_per_cta=W, ctas_per_slice=1, threads_per_cta=256, flags=CO,
                               **kw)
    for h in (ht, hr):
        mcinv.mcinv_set_trace_weights(h, q)
        mcinv.mcinv_burnin(h, 10)
        mcinv.mcinv_sample(h, 32)
    dt, st = mcinv.mcinv_estimate(ht, mcinv.MCINV_EST_DIAG)
    dr, sr = mcinv.mcinv_estimate(hr, mcinv.MCINV_EST_DIAG)
    assert np.array_equal(dt, dr) and np.array_equal(st, sr)
    tt_, _ = mcinv.mcinv_estimate(ht, mcinv.MCINV_EST_TRACE, q_diag=q)
    tr_, _ = mcinv.mcinv_estimate(hr, mcinv.MCINV_EST_TRACE, q_diag=q)
    assert np.array_equal(tt_, tr_)
    bt, _ = mcinv.mcinv_estimate(ht, mcinv.MCINV_EST_BLOCK)
    br, _ = mcinv.mcinv_estimate(hr, mcinv.MCINV_EST_BLOCK)
    assert np.array_equal(bt, br)  # the same BF16 shadows, the same contraction
    tt = mcinv.mcinv_trace_series(ht)
    tr = mcinv.mcinv_trace_series(hr)
    # FP32 per-warp partials summed over other warps: the same terms, another order
    assert len(tt) == 32 and np.abs(tt - tr).max() <= 1e-5 * np.abs(tr).max()
    for h in (ht, hr):
        mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("make,K", [(lambda: wl.u1_lattice((32, 16), 0.12, 0.08, seed=10), 64),
                                    (lambda: _real(wl.u1_lattice((16, 16), 0.12, 0.08, seed=11)), 64)])
def test_wave_follows_the_oracle_for_100_cycles(make, K):
    """Same-draw trajectories of C' = P C P^T (P: the greedy colouring of the test
    helper, written apart from the library's) against the oracle after 20 and 100
    cycles, 1e-4 relative; 100 cycles are 12 launches of 8 and one of 4."""
    c = make()
    h = mcinv.create_from_csr(c, K=K, seed=8, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=8, flags=WAVE | CO)
    assert mcinv.mcinv_info(h)["sweep_kernel"] == 6
    o, _ = greedy_order(c)
    cref = permuted(c, o)
    done = 0
    for cyc in (20, 100):
        mcinv.mcinv_burnin(h, cyc - done)
        done = cyc
        z, w, got = mcinv.mcinv_get_state(h)
        assert got == cyc
        st, _, _ = oracle.run(cref, K, seed=8, ncycles=cyc, diag=False)
        zo, wo = (st.z, st.w) if c.is_complex else (st.z.real, st.w.real)
        assert np.abs(z[o] - zo).max() <= 1e-4 * np.abs(zo).max(), cyc
        assert np.abs(w[o] - wo).max() <= 1e-4 * np.abs(wo).max(), cyc
    mcinv.mcinv_destroy(h)


def test_wave_many_cycles_in_one_launch():
    """64 cycles in one launch against the chain-sliced kernel."""
    c = wl.u1_lattice((16, 16), 0.12, 0.08, seed=12)
    hw = mcinv.create_from_csr(c, K=256, seed=3, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=64, flags=WAVE | CO)
    hr = mcinv.create_from_csr(c, K=256, seed=3, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=64, chains_per_cta=64,
                               ctas_per_slice=1, threads_per_cta=256, flags=CO)
    for h in (hw, hr):
        mcinv.mcinv_burnin(h, 64)
    zw, ww, _ = mcinv.mcinv_get_state(hw)
    zr, wr, _ = mcinv.mcinv_get_state(hr)
    assert np.array_equal(zw, zr) and np.array_equal(ww, wr)
    for h in (hw, hr):
        mcinv.mcinv_destroy(h)


def test_wave_rejections():
    # a random pattern has many levels; the 16^4 lattice's band (4096 positions) does not fit
    for c in (wl.pedigree(3000, 1.2, 1), wl.u1_lattice((16, 16, 16, 16), 0.06, 0.04, seed=1)):
        with pytest.raises(mcinv.McinvError) as e:
            mcinv.create_from_csr(c, K=64, flags=WAVE | CO)
        assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    with pytest.raises(mcinv.McinvError) as e:  # the given order of a lattice: many levels
        mcinv.create_from_csr(wl.u1_lattice((8, 8), 0.1, 0.1, seed=1), K=64, flags=WAVE)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    for extra in (mcinv.MCINV_F_GRID_NOPAIR, mcinv.MCINV_F_GRID_TILE):
        with pytest.raises(mcinv.McinvError) as e:
            mcinv.create_from_csr(wl.u1_lattice((8, 8), 0.1, 0.1, seed=1), K=64, flags=WAVE | CO | extra)
        assert e.value.status == mcinv.MCINV_E_ARG


def test_wave_trace_series_without_the_diagonal():
    """Trace weights with MCINV_F_NO_DIAG: the epilogue forms z conj(w) for the trace alone."""
    c = wl.u1_lattice((16, 16), 0.12, 0.08, seed=15)
    q = wl.q_diag(c.n, 2)
    nd = mcinv.MCINV_F_NO_DIAG
    series = []
    for flags, kw in ((WAVE | CO | nd, {}), (CO | nd, dict(chains_per_cta=64, ctas_per_slice=1, threads_per_cta=256))):
        h = mcinv.create_from_csr(c, K=512, seed=2, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=8, flags=flags, **kw)
        if flags & mcinv.MCINV_F_GRID_WAVE:
            assert mcinv.mcinv_info(h)["sweep_kernel"] == 6
        mcinv.mcinv_set_trace_weights(h, q)
        mcinv.mcinv_burnin(h, 10)
        mcinv.mcinv_sample(h, 32)
        series.append(mcinv.mcinv_trace_series(h))
        mcinv.mcinv_destroy(h)
    tw, tr = series
    assert len(tw) == 32 and np.abs(tw - tr).max() <= 1e-5 * np.abs(tr).max()


def test_wave_expired_wait_ends_the_launch_and_the_context_stays_usable():
    """MCINV_F_TEST_EXPIRE_WAIT: a stage announced to its mbarrier and never copied. Every
    CTA's bounded wait (2 s) expires, the launch ends without touching shared memory it did
    not fill, and mcinv_sync reports MCINV_E_TIMEOUT; kernels then run as before."""
    import time
    c = wl.u1_lattice((16, 16), 0.12, 0.08, seed=16)
    h = mcinv.create_from_csr(c, K=64, seed=1, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=2,
                              flags=WAVE | CO | mcinv.MCINV_F_TEST_EXPIRE_WAIT)
    t0 = time.time()
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_burnin(h, 2)
        mcinv.mcinv_sync(h)
    assert e.value.status == mcinv.MCINV_E_TIMEOUT
    assert time.time() - t0 < 60
    mcinv.mcinv_destroy(h)
    _pair(c, 64, 4, cycles=(1, 3))
    with pytest.raises(mcinv.McinvError) as e:  # the hook is for the wavefront sweep only
        mcinv.create_from_csr(c, K=64, flags=CO | mcinv.MCINV_F_TEST_EXPIRE_WAIT)
    assert e.value.status == mcinv.MCINV_E_ARG
