"""The tile-staged sweep (sweep_tiled.cu): a CTA stages a tile's distinct neighbours
in shared memory once and updates the tile's rows from there.  Its arithmetic is
every other kernel's, so the chains must equal the chain-sliced kernel's bit for
bit: on 2D and 4D U(1) lattices in the colour order (complex), on a real matrix of
the same pattern, with a ragged last chain block, and with the estimates (diagonal
partials, trace series, BF16 shadows of a block) accumulated while sampling."""
import numpy as np
import pytest

from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TILE = mcinv.MCINV_F_GRID | mcinv.MCINV_F_GRID_BULK | mcinv.MCINV_F_GRID_TILE
CO = mcinv.MCINV_F_COLOR_ORDER


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def _real(c):
    """The same pattern with the real parts (a real non-symmetric, structurally symmetric C)."""
    return wl.CSR(c.n, c.row_ptr, c.col, np.ascontiguousarray(c.val.real))


def _pair(c, K, cycles=(1, 6, 20)):
    W = 64 if np.iscomplexobj(c.val) else 128
    ht = mcinv.create_from_csr(c, K=K, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, flags=TILE | CO)
    hr = mcinv.create_from_csr(c, K=K, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, chains_per_cta=W, ctas_per_slice=1,
                               threads_per_cta=256, flags=CO)
    info = mcinv.mcinv_info(ht)
    assert info["sweep_kernel"] == 5 and info["grid_ctas"] >= 1 and info["threads_per_cta"] == 512
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


@pytest.mark.parametrize("K", [130, 520])
@pytest.mark.parametrize("make", [lambda: wl.u1_lattice((16, 16), 0.12, 0.08, seed=2),
                                  lambda: wl.u1_lattice((24, 20), 0.12, 0.08, seed=3),
                                  lambda: _real(wl.u1_lattice((20, 16), 0.12, 0.08, seed=4)),
                                  lambda: wl.u1_lattice((4, 6, 4, 4), 0.06, 0.04, seed=5)])
def test_tiled_sweep_equals_chain_sliced_kernel(make, K):
    c = make()
    # real: K a multiple of 4 (132 or 520: 33 or 130 vectors, the last 32-vector block ragged)
    _pair(c, K if np.iscomplexobj(c.val) else K + (-K) % 4)


@pytest.mark.parametrize("make", [lambda: wl.u1_lattice((16, 16), 0.12, 0.08, seed=6),
                                  lambda: _real(wl.u1_lattice((16, 12), 0.12, 0.08, seed=7))])
def test_tiled_estimates_equal_chain_sliced_kernel(make):
    c = make()
    q = wl.q_diag(c.n, 1)
    W = 64 if np.iscomplexobj(c.val) else 128
    kw = dict(acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=8, block_rows=np.arange(c.n), block_cols=np.arange(64))
    ht = mcinv.create_from_csr(c, K=512, seed=2, flags=TILE | CO, **kw)
    hr = mcinv.create_from_csr(c, K=512, seed=2, chains_per_cta=W, ctas_per_slice=1, threads_per_cta=256, flags=CO,
                               **kw)
    for h in (ht, hr):
        mcinv.mcinv_set_trace_weights(h, q)
        mcinv.mcinv_burnin(h, 10)
        mcinv.mcinv_sample(h, 32)
    dt, st = mcinv.mcinv_estimate(ht, mcinv.MCINV_EST_DIAG)
    dr, sr = mcinv.mcinv_estimate(hr, mcinv.MCINV_EST_DIAG)
    assert np.array_equal(dt, dr) and np.array_equal(st, sr)
    bt, _ = mcinv.mcinv_estimate(ht, mcinv.MCINV_EST_BLOCK)
    br, _ = mcinv.mcinv_estimate(hr, mcinv.MCINV_EST_BLOCK)
    assert np.array_equal(bt, br)  # the same BF16 shadows, the same contraction
    tt = mcinv.mcinv_trace_series(ht)
    tr = mcinv.mcinv_trace_series(hr)
    # FP32 per-warp partials summed over other warps: the same terms, another order
    assert len(tt) == 32 and np.abs(tt - tr).max() <= 1e-5 * np.abs(tr).max()
    for h in (ht, hr):
        mcinv.mcinv_destroy(h)


def test_tiled_sweep_rejections():
    # a random pattern: every tile names far more neighbours than the stage holds
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.create_from_csr(wl.pedigree(3000, 1.2, 1), K=64, flags=TILE | CO)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    with pytest.raises(mcinv.McinvError) as e:  # the tiled form is on the pair layout
        mcinv.create_from_csr(wl.u1_lattice((8, 8), 0.1, 0.1, seed=1), K=64, flags=TILE | mcinv.MCINV_F_GRID_NOPAIR)
    assert e.value.status == mcinv.MCINV_E_ARG
