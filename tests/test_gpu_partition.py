"""The block partition of Sec. 4 on the GPU (mcinv_create_partitioned): the
device sweeps C~ = S^-1 C S^-1 and maps z = S^-1 z~, w = S^-H w~, so its chains
must follow the oracle's block sweep of C draw for draw, and its diagonal and
trace must estimate C^-1 where the scalar sweep cannot even start."""
import numpy as np
import pytest

import oracle
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl
from test_block_partition_pins import zero_diagonal_pairs

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def mixed_blocks(nblocks, seed, complex_=False):
    """Blocks of 1, 2 or 3 rows: one-row blocks with a dominant diagonal, two-row blocks
    [[0, a], [b, 0]] with ab < 0 (zero diagonal), three-row blocks 2 I + a random 0.4 part;
    weak couplings between blocks."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice([1, 2, 3], nblocks)
    bp = np.concatenate([[0], np.cumsum(sizes)])
    n = int(bp[-1])
    a = np.zeros((n, n), dtype=np.complex128 if complex_ else np.float64)
    for b in range(nblocks):
        r = slice(bp[b], bp[b + 1])
        if sizes[b] == 1:
            a[r, r] = rng.uniform(1.5, 2.5) * rng.choice([-1, 1])
        elif sizes[b] == 2:
            s = rng.choice([-1, 1])
            a[bp[b], bp[b] + 1] = rng.uniform(1, 2) * s
            a[bp[b] + 1, bp[b]] = -rng.uniform(1, 2) * s
        else:
            a[r, r] = 2 * np.eye(3) + 0.4 * rng.uniform(-1, 1, (3, 3))
    blk = np.repeat(np.arange(nblocks), sizes)
    for i in range(n):
        for j in rng.choice(n, 3, replace=False):
            if blk[j] != blk[i]:
                v = 0.1 * rng.uniform(-1, 1)
                a[i, j] += v * np.exp(1j * rng.uniform(0, 2 * np.pi)) if complex_ else v
    rows, cols = np.nonzero(a)
    return wl.csr_from_coo(n, rows, cols, a[rows, cols]), bp


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("make,K,shape", [
    (lambda: zero_diagonal_pairs(40, 3), 32, {}),
    (lambda: zero_diagonal_pairs(40, 4, True), 24, {}),
    (lambda: mixed_blocks(60, 5), 40, {"chains_per_cta": 8, "threads_per_cta": 128}),
    (lambda: mixed_blocks(60, 6, True), 16, {"chains_per_cta": 16, "threads_per_cta": 256, "ctas_per_slice": 2}),
])
def test_trajectory_is_the_oracle_block_sweep(make, K, shape):
    c, bp = make()
    h = mcinv.create_from_csr(c, K=K, seed=7, acc=mcinv.MCINV_ACC_FP32_SIMT, partition=bp, **shape)
    st, done = None, 0
    for cyc in (1, 10, 40):
        mcinv.mcinv_burnin(h, cyc - done)
        st = oracle.run_block(c, bp, K, seed=7, cycle0=done, ncycles=cyc - done, state=st)
        done = cyc
        z, w, _ = mcinv.mcinv_get_state(h)
        assert _rel(z, st.z) <= TOL and _rel(w, st.w) <= TOL, (cyc, _rel(z, st.z), _rel(w, st.w))
    mcinv.mcinv_destroy(h)


@pytest.mark.parametrize("complex_,flags", [(False, 0), (True, 0), (False, mcinv.MCINV_F_COLOR_ORDER),
                                            (True, mcinv.MCINV_F_COLOR_ORDER)])
def test_diagonal_trace_and_block_estimate_the_inverse(complex_, flags):
    c, bp = mixed_blocks(90, 9, complex_)
    inv = np.linalg.inv(c.to_dense())
    one = np.array([bp[b] for b in range(len(bp) - 1) if bp[b + 1] - bp[b] == 1])
    R, S = one[::2], one[1::3]
    h = mcinv.create_from_csr(c, K=256, seed=3, acc=mcinv.MCINV_ACC_FP32_SIMT, batch_cycles=8, flags=flags,
                              partition=bp, block_rows=R, block_cols=S)
    mcinv.mcinv_burnin(h, 40)
    mcinv.mcinv_sample(h, 240)
    d, dse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_DIAG)
    q = wl.q_diag(c.n, 1)
    tr, tse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_TRACE, q_diag=q)
    b, bse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
    mcinv.mcinv_destroy(h)
    re = (lambda x: x.real) if complex_ else (lambda x: x)
    for est, se, truth in ((d, dse, np.diag(inv)), (b, bse, inv[np.ix_(R, S)])):
        z = np.abs(re(est) - re(truth)).ravel() / re(se).ravel()
        assert (z > 3.5).mean() < 0.02 and 0.7 < np.sqrt(np.mean(z ** 2)) < 1.35
    assert abs(re(tr) - re((q * np.diag(inv)).sum())) < 4 * re(tse)


def test_one_row_partition_is_the_plain_sampler():
    c = wl.random_dominant(300, 4, 1.4, 5)
    h1 = mcinv.create_from_csr(c, K=64, seed=2, acc=mcinv.MCINV_ACC_FP32_SIMT, partition=np.arange(c.n + 1))
    h2 = mcinv.create_from_csr(c, K=64, seed=2, acc=mcinv.MCINV_ACC_FP32_SIMT)
    mcinv.mcinv_burnin(h1, 20)
    mcinv.mcinv_burnin(h2, 20)
    z1, w1, _ = mcinv.mcinv_get_state(h1)
    z2, w2, _ = mcinv.mcinv_get_state(h2)
    assert np.array_equal(z1, z2) and np.array_equal(w1, w2)


def test_state_round_trip():
    c, bp = mixed_blocks(50, 11, True)
    h = mcinv.create_from_csr(c, K=32, seed=4, acc=mcinv.MCINV_ACC_FP32_SIMT, partition=bp)
    mcinv.mcinv_burnin(h, 9)
    z, w, cyc = mcinv.mcinv_get_state(h)
    mcinv.mcinv_burnin(h, 6)
    z1, w1, _ = mcinv.mcinv_get_state(h)
    h2 = mcinv.create_from_csr(c, K=32, seed=4, acc=mcinv.MCINV_ACC_FP32_SIMT, partition=bp)
    mcinv.mcinv_set_state(h2, z, w, cyc)
    mcinv.mcinv_burnin(h2, 6)
    z2, w2, _ = mcinv.mcinv_get_state(h2)
    assert _rel(z2, z1) < 1e-5 and _rel(w2, w1) < 1e-5


def test_rejections():
    c, bp = zero_diagonal_pairs(10, 2)
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.create_from_csr(c, K=8, partition=np.arange(c.n + 1))  # zero diagonal, one-row blocks
    assert e.value.status == mcinv.MCINV_E_SINGULAR_DIAG
    bad = wl.csr_from_coo(2, [0, 1], [1, 0], np.array([1.0, 2.0]))  # eigenvalues +-sqrt(2)
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.create_from_csr(bad, K=8, partition=np.array([0, 2]))
    assert e.value.status == mcinv.MCINV_E_SINGULAR_DIAG
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.create_from_csr(c, K=8, partition=np.array([0, 3, c.n]))  # block of 17 rows
    assert e.value.status == mcinv.MCINV_E_ARG
    h = mcinv.create_from_csr(c, K=8, partition=bp)
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_set_trace_weights(h, np.ones(c.n))
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.create_from_csr(c, K=8, partition=bp, block_rows=np.array([0]), block_cols=np.array([1]))
    assert e.value.status == mcinv.MCINV_E_UNSUPPORTED
