"""The grid-wide sweep (MCINV_F_GRID): one cooperative launch in which a warp
updates one row for 32 x V chains and all CTAs share every dependency level, with
a grid barrier between levels.  Its arithmetic is the chain-sliced kernel's in the
same order, so with 32 x V-chain slices (the same diagonal units) the chains, the
diagonal and the tensor-core block must equal that kernel's bit for bit, in either
sweep order, for real and complex matrices, and follow the oracle."""
import numpy as np
import pytest

import oracle
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GR = mcinv.MCINV_F_GRID
GB = mcinv.MCINV_F_GRID | mcinv.MCINV_F_GRID_BULK
GBS = GB | mcinv.MCINV_F_GRID_NOPAIR  # bulk staging, z and w in separate buffers
GP = GB | mcinv.MCINV_F_GRID_PAIR  # bulk staging on the pair layout, in the shape threads names
CO = mcinv.MCINV_F_COLOR_ORDER


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def _pair(c, K, flags=0, cycles=(1, 7, 25), threads=384, grid=GR, **kw):
    W = 64 if c.is_complex else 128
    # threads 0: the kernel's own (bulk staging: the pair layout where C is structurally symmetric)
    hg = mcinv.create_from_csr(c, K=K, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, threads_per_cta=threads,
                               flags=flags | grid, **kw)
    hr = mcinv.create_from_csr(c, K=K, seed=5, acc=mcinv.MCINV_ACC_FP32_SIMT, chains_per_cta=W, ctas_per_slice=1,
                               threads_per_cta=256, flags=flags, **kw)
    info = mcinv.mcinv_info(hg)
    # the pair layout where C is structurally symmetric (bulk staging, default threads)
    want = (3, 4) if grid == GB and threads == 0 else (4,) if grid == GP else (3,) if grid in (GB, GBS) else (2,)
    assert info["sweep_kernel"] in want and info["grid_ctas"] >= 1
    done = 0
    for cyc in cycles:
        for h in (hg, hr):
            mcinv.mcinv_burnin(h, cyc - done)
        done = cyc
        zg, wg, _ = mcinv.mcinv_get_state(hg)
        zr, wr, _ = mcinv.mcinv_get_state(hr)
        assert np.array_equal(zg, zr) and np.array_equal(wg, wr), cyc
    return hg, hr


@pytest.mark.parametrize("flags", [0, CO])
@pytest.mark.parametrize("K,threads,grid", [(256, 384, GR), (200, 512, GR), (36, 384, GR), (256, 0, GB),
                                            (200, 0, GB), (36, 0, GB), (256, 384, GB), (200, 0, GBS),
                                            (1024, 192, GB), (520, 192, GB), (1024, 96, GB), (900, 96, GB),
                                            (36, 96, GB), (256, 512, GB), (200, 512, GBS), (36, 512, GBS),
                                            (256, 512, GP), (200, 384, GP), (36, 384, GP), (1024, 384, GP),
                                            (520, 256, GP), (900, 256, GP)])
def test_grid_equals_chain_sliced_kernel_real(flags, K, threads, grid):
    c = wl.pedigree(6000, 1.2, 3)  # long rows (pieces), 60-odd levels in the given order
    hg, hr = _pair(c, K, flags=flags, threads=threads, grid=grid)
    for h in (hg, hr):
        mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("grid,threads", [(GR, 384), (GB, 0), (GBS, 0), (GB, 192), (GB, 96), (GBS, 512), (GP, 512),
                                          (GP, 384), (GP, 256)])
@pytest.mark.parametrize("flags", [0, CO])
def test_grid_equals_chain_sliced_kernel_complex(flags, grid, threads):
    c = wl.u1_lattice((16, 16), 0.12, 0.08, seed=2)
    hg, hr = _pair(c, 130 if threads in (0, 384) else 520, flags=flags, grid=grid, threads=threads)
    for h in (hg, hr):
        mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("threads", [384, 256])
def test_pair_shapes_on_a_4d_lattice(threads):
    # 8 neighbours a row: one row in flight a warp (9 or 13 slots)
    c = wl.u1_lattice((4, 6, 4, 4), 0.06, 0.04, seed=3)
    hg, hr = _pair(c, 520, flags=CO, cycles=(2, 9), grid=GP, threads=threads)
    for h in (hg, hr):
        mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("grid,threads", [(GR, 384), (GB, 0), (GBS, 0), (GB, 96), (GBS, 512)])
def test_grid_equals_chain_sliced_kernel_wilson_dirac(grid, threads):
    c = wl.wilson_dirac((3, 3, 3, 4), 0.1)  # 4 x 4 spinor hops, 14 nonzeros per row
    hg, hr = _pair(c, 64 if threads in (0, 384) else 320, flags=CO, cycles=(3, 12), grid=grid, threads=threads)
    for h in (hg, hr):
        mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("grid,threads", [(GR, 384), (GB, 0), (GBS, 0), (GB, 192), (GB, 96), (GBS, 512), (GP, 512),
                                          (GP, 256)])
@pytest.mark.parametrize("flags", [0, CO])
def test_grid_estimates_equal_chain_sliced_kernel(flags, grid, threads):
    c = wl.pedigree(3000, 1.2, 7)
    q = wl.q_diag(c.n, 1)
    kw = dict(acc=mcinv.MCINV_ACC_BF16_TC, batch_cycles=8, block_rows=np.arange(c.n), block_cols=np.arange(256))
    hg = mcinv.create_from_csr(c, K=512, seed=2, flags=flags | grid, threads_per_cta=threads, **kw)
    hr = mcinv.create_from_csr(c, K=512, seed=2, chains_per_cta=128, ctas_per_slice=1, threads_per_cta=256,
                               flags=flags, **kw)
    for h in (hg, hr):
        mcinv.mcinv_set_trace_weights(h, q)
        mcinv.mcinv_burnin(h, 10)
        mcinv.mcinv_sample(h, 32)
    dg, sg = mcinv.mcinv_estimate(hg, mcinv.MCINV_EST_DIAG)
    dr, sr = mcinv.mcinv_estimate(hr, mcinv.MCINV_EST_DIAG)
    assert np.array_equal(dg, dr) and np.array_equal(sg, sr)
    bg, _ = mcinv.mcinv_estimate(hg, mcinv.MCINV_EST_BLOCK)
    br, _ = mcinv.mcinv_estimate(hr, mcinv.MCINV_EST_BLOCK)
    assert np.array_equal(bg, br)  # same BF16 shadows, same contraction
    tg = mcinv.mcinv_trace_series(hg)
    tr = mcinv.mcinv_trace_series(hr)
    # FP32 per-warp partials summed over other warps: same terms, another order
    assert len(tg) == 32 and np.abs(tg - tr).max() <= 1e-5 * np.abs(tr).max()
    for h in (hg, hr):
        mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("grid", [GR, GB])
@pytest.mark.parametrize("case", ["pedigree", "lattice"])
def test_grid_follows_the_oracle(case, grid):  # the default thread count, 384
    if case == "pedigree":
        c, K, cyc = wl.pedigree(2000, 1.2, 11), 64, 30
    else:
        c, K, cyc = wl.u1_lattice((12, 12), 0.12, 0.08, seed=4), 34, 40
    h = mcinv.create_from_csr(c, K=K, seed=8, acc=mcinv.MCINV_ACC_FP32_SIMT, flags=grid)
    mcinv.mcinv_burnin(h, cyc)
    z, w, got = mcinv.mcinv_get_state(h)
    st, _, _ = oracle.run(c, K, seed=8, ncycles=cyc)
    assert got == cyc
    assert np.abs(z - (st.z if c.is_complex else st.z.real)).max() <= 1e-4 * np.abs(st.z).max()
    assert np.abs(w - (st.w if c.is_complex else st.w.real)).max() <= 1e-4 * np.abs(st.w).max()
    mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("grid", [GR, GB])
def test_grid_many_cycles_in_one_launch(grid):
    # 64 cycles x 2 levels of grid barriers in one launch, then against the oracle
    c = wl.u1_lattice((8, 8), 0.12, 0.08, seed=6)
    h = mcinv.create_from_csr(c, K=64, seed=3, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=64, flags=grid | CO)
    mcinv.mcinv_burnin(h, 64)
    z, w, _ = mcinv.mcinv_get_state(h)
    order, _ = mcinv.mcinv_color_order(c.n, c.row_ptr, c.col)
    inv = np.empty(c.n, dtype=np.int64)
    inv[order] = np.arange(c.n)
    rows = np.repeat(np.arange(c.n), np.diff(c.row_ptr))
    cp = wl.csr_from_coo(c.n, inv[rows], inv[c.col], c.val)
    st, _, _ = oracle.run(cp, 64, seed=3, ncycles=64)
    assert np.abs(z[order] - st.z).max() <= 1e-4 * np.abs(st.z).max()
    assert np.abs(w[order] - st.w).max() <= 1e-4 * np.abs(st.w).max()
    mcinv.mcinv_destroy(h)


def test_grid_rejections():
    c = wl.random_dominant(100, 4, 1.5, 1)
    with pytest.raises(mcinv.McinvError) as e:  # K not a multiple of 4 chains per lane
        mcinv.create_from_csr(c, K=30, flags=GR)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    with pytest.raises(mcinv.McinvError) as e:  # 256 threads
        mcinv.create_from_csr(c, K=64, threads_per_cta=256, flags=GR)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    with pytest.raises(mcinv.McinvError) as e:  # bulk staging with 256 threads (96, 192, 384 or 512)
        mcinv.create_from_csr(c, K=64, threads_per_cta=256, flags=GB)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    for flags, threads in ((GP, 192), (GP | mcinv.MCINV_F_GRID_NOPAIR, 384), (GR | mcinv.MCINV_F_GRID_PAIR, 384)):
        with pytest.raises(mcinv.McinvError) as e:  # the pair shapes: 512, 384 or 256 threads, bulk staging
            mcinv.create_from_csr(wl.pedigree(500, 1.2, 1), K=64, threads_per_cta=threads, flags=flags)
        assert e.value.status == mcinv.MCINV_E_ARG
    with pytest.raises(mcinv.McinvError) as e:  # the pair layout of a matrix that is not structurally symmetric
        mcinv.create_from_csr(c, K=64, threads_per_cta=384, flags=GP)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    with pytest.raises(mcinv.McinvError) as e:  # and the staged kernel
        mcinv.create_from_csr(c, K=64, flags=GR | mcinv.MCINV_F_STAGED, chains_per_cta=32)
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED


def test_pair_layout_is_used_and_survives_state_round_trips():
    # a structurally symmetric matrix runs on the pair layout; reading the state
    # between launches, writing it back and resuming give the uninterrupted run's bits
    c = wl.pedigree(4000, 1.2, 9)
    h = mcinv.create_from_csr(c, K=256, seed=6, acc=mcinv.MCINV_ACC_FP32_SIMT, flags=GB | CO, batch_cycles=3)
    info = mcinv.mcinv_info(h)
    assert info["sweep_kernel"] == 4 and info["threads_per_cta"] == 384  # 12 warps, two blocks a warp
    g = mcinv.create_from_csr(c, K=256, seed=6, acc=mcinv.MCINV_ACC_FP32_SIMT, flags=GBS | CO, batch_cycles=3)
    assert mcinv.mcinv_info(g)["sweep_kernel"] == 3
    mcinv.mcinv_burnin(h, 7)
    z, w, cyc = mcinv.mcinv_get_state(h)
    mcinv.mcinv_set_state(h, z, w, cyc)
    mcinv.mcinv_burnin(h, 5)
    mcinv.mcinv_burnin(g, 12)
    zh, wh, _ = mcinv.mcinv_get_state(h)
    zg, wg, _ = mcinv.mcinv_get_state(g)
    assert np.array_equal(zh, zg) and np.array_equal(wh, wg)
    # a matrix that is not structurally symmetric keeps separate buffers
    r = wl.random_dominant(300, 4, 1.5, 2)
    hr = mcinv.create_from_csr(r, K=64, flags=GB)
    assert mcinv.mcinv_info(hr)["sweep_kernel"] == 3
    for x in (h, g, hr):
        mcinv.mcinv_destroy(x)


@pytest.mark.parametrize("grid,threads", [(GR, 384), (GB, 0), (GBS, 384), (GBS, 512), (GP, 256)])
@pytest.mark.parametrize("batch", [1, 8])
def test_grid_reports_divergence(grid, threads, batch):
    """C = [[1, 3], [4, 1]]: sp(T) > 1, the chains blow up (Sec. 2.2).  The grid-wide sweep
    checks the bound on each launch's last cycle; a diverging chain is still beyond it there."""
    csr = wl.csr_from_coo(2, [0, 0, 1, 1], [0, 1, 0, 1], np.array([1.0, 3.0, 4.0, 1.0]))
    h = mcinv.create_from_csr(csr, K=8, seed=1, acc=mcinv.MCINV_ACC_FP32_SIMT, flags=grid, threads_per_cta=threads,
                              batch_cycles=batch)
    mcinv.mcinv_burnin(h, 64)
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_sync(h)
    assert e.value.status == mcinv.MCINV_E_DIVERGED
    mcinv.mcinv_destroy(h)
