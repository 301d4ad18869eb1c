"""The pool: many real matrices advanced together by persistent kernels that
read device tables (the batched form), with members joining and leaving
between steps (continuous batching).

Checks: every member's chains follow the FP64 oracle (same draws: the matrix
id keys the noise); a member's results are bit-identical whether it runs
alone or alongside others that join later; its full inverse equals the
single-matrix handle's; admission refuses what does not fit in the arena
and accepts it after a release; the batch estimates cover the dense inverse.
"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(__file__))
import oracle  # noqa: E402
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def run_until_done(pool, tickets, max_steps=10_000):
    for _ in range(max_steps):
        if all(mcinv.mcinv_pool_poll(pool, t) for t in tickets):
            return
        mcinv.mcinv_pool_step(pool)
    raise AssertionError("pool did not finish")


def test_pool_members_follow_the_oracle():
    K, B, burn, samp = 64, 4, 6, 7
    mats = [wl.random_dominant(n, 4, 1.5, seed) for n, seed in ((64, 1), (200, 2), (517, 3))]
    pool = mcinv.mcinv_pool_create(K=K, seed=11, mem_budget=1 << 28, max_slots=8, batch_cycles=B)
    tickets = [mcinv.mcinv_pool_submit(pool, c, matrix_id=100 + k, burnin=burn, samples=samp, want_inverse=True)
               for k, c in enumerate(mats)]
    run_until_done(pool, tickets)
    for k, (c, t) in enumerate(zip(mats, tickets)):
        z, w, cyc = mcinv.mcinv_pool_get_state(pool, t, c.n)
        assert cyc == burn + samp
        st, dacc, _ = oracle.run(c, K, seed=11, matrix=100 + k, ncycles=burn + samp, acc_from=burn)
        assert rel_err(z, st.z.real) < TOL and rel_err(w, st.w.real) < TOL
        dm, _ = mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_DIAG, c.n)
        assert rel_err(dm, dacc.sum(0).real / (K * samp)) < TOL
    info = mcinv.mcinv_pool_info(pool)
    assert info["active"] == 3 and info["kernel_launches"] >= 4


def test_pool_result_is_the_same_alone_and_in_the_mix():
    K, B = 64, 4
    a = wl.random_dominant(300, 4, 1.5, 7)
    others = [wl.random_dominant(n, 4, 1.5, 20 + n) for n in (90, 640, 150)]

    alone = mcinv.mcinv_pool_create(K=K, seed=3, mem_budget=1 << 28, max_slots=8, batch_cycles=B)
    ta = mcinv.mcinv_pool_submit(alone, a, matrix_id=5, burnin=9, samples=23)
    run_until_done(alone, [ta])
    ref = {k: mcinv.mcinv_pool_estimate(alone, ta, k, a.n) for k in (mcinv.MCINV_EST_DIAG, mcinv.MCINV_EST_BLOCK)}

    mix = mcinv.mcinv_pool_create(K=K, seed=3, mem_budget=1 << 28, max_slots=8, batch_cycles=B)
    t0 = mcinv.mcinv_pool_submit(mix, others[0], matrix_id=1, burnin=3, samples=5)
    mcinv.mcinv_pool_step(mix)
    tm = mcinv.mcinv_pool_submit(mix, a, matrix_id=5, burnin=9, samples=23)  # joins while others run
    mcinv.mcinv_pool_step(mix)
    t1 = mcinv.mcinv_pool_submit(mix, others[1], matrix_id=2, burnin=11, samples=40)
    mcinv.mcinv_pool_step(mix)
    run_until_done(mix, [t0])
    mcinv.mcinv_pool_release(mix, t0)  # leaves; its memory is reused by the next member
    t2 = mcinv.mcinv_pool_submit(mix, others[2], matrix_id=3, burnin=2, samples=30)
    run_until_done(mix, [tm, t1, t2])
    for k, (m, se) in ref.items():
        m2, se2 = mcinv.mcinv_pool_estimate(mix, tm, k, a.n)
        assert np.array_equal(m, m2) and np.array_equal(se, se2, equal_nan=True), k


def test_pool_full_inverse_equals_single_handle():
    # one step's product a batch (fold_steps 1), as the handle folds every batch
    K, B, burn, samp = 128, 4, 8, 16
    c = wl.random_dominant(256, 4, 1.5, 0)
    pool = mcinv.mcinv_pool_create(K=K, seed=9, mem_budget=1 << 28, max_slots=4, batch_cycles=B, fold_steps=1)
    t = mcinv.mcinv_pool_submit(pool, c, matrix_id=4, burnin=burn, samples=samp)
    run_until_done(pool, [t])
    pm, pse = mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_BLOCK, c.n)
    R = np.arange(c.n)
    h = mcinv.create_from_csr(c, K=K, seed=9, matrix_id=4, batch_cycles=B, acc=mcinv.MCINV_ACC_BF16_TC,
                              block_rows=R, block_cols=R)
    mcinv.mcinv_burnin(h, burn)
    mcinv.mcinv_sample(h, samp)
    hm, hse = mcinv.mcinv_estimate(h, mcinv.MCINV_EST_BLOCK)
    assert np.abs(pm - hm).max() <= 1e-12 * np.abs(hm).max()
    assert np.abs(pse - hse).max() <= 1e-9 * np.abs(hse).max()


@pytest.mark.parametrize("F", [1, 3])
def test_pool_folded_batches_follow_the_oracle(F):
    """The block products of F sampling steps summed in FP32 by the contraction's
    epilogue and folded once (the batch-means SE over batches of F steps' sampling
    cycles): mean and SE of each member's full inverse equal the oracle's from the same
    draws, its states rounded to the BF16 operands, within 1e-4 of the largest entry of
    the mean.  Burn-ins that end inside a step give a short first batch.

    The SE shares the mean's absolute bar: the GPU rounds its FP32 states to BF16 and
    the oracle its FP64 states, so a value within ~1e-7 of a rounding boundary lands on
    the other BF16 neighbour (one operand off by 2^-7 of itself), which moves a batch
    mean by about 1e-5 of the largest entry; the SE, a spread of batch means ~20 times
    smaller than the mean, takes that absolute error, not 1e-4 of itself."""
    import _block_oracle
    K, B = 64, 4
    mats = [(wl.random_dominant(n, 4, 1.5, seed), burn, samp)
            for n, seed, burn, samp in ((130, 1, 6, 33), (300, 2, 4, 16), (77, 3, 9, 50))]
    pool = mcinv.mcinv_pool_create(K=K, seed=17, mem_budget=1 << 28, max_slots=4, batch_cycles=B, fold_steps=F)
    assert mcinv.mcinv_pool_info(pool)["fold_steps"] == F
    tickets = [mcinv.mcinv_pool_submit(pool, c, matrix_id=40 + k, burnin=burn, samples=samp)
               for k, (c, burn, samp) in enumerate(mats)]
    run_until_done(pool, tickets)
    for k, ((c, burn, samp), t) in enumerate(zip(mats, tickets)):
        m, se = mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_BLOCK, c.n)
        om, ose = _block_oracle.block_estimate(c, K, 17, 40 + k, burn, samp, B, F)
        bar = 1e-4 * np.abs(om).max()
        assert np.abs(m - om).max() <= bar and np.abs(se - ose).max() <= bar, \
            (F, k, rel_err(m, om), np.abs(se - ose).max() / np.abs(om).max())
    mcinv.mcinv_pool_destroy(pool)


def test_pool_admission_by_device_memory():
    c = wl.random_dominant(1024, 4, 1.5, 5)
    probe = mcinv.mcinv_pool_create(K=64, mem_budget=1 << 24, max_slots=4)
    need = mcinv.mcinv_pool_footprint(probe, c.n, c.nnz, True)
    pool = mcinv.mcinv_pool_create(K=64, mem_budget=int(need * 1.5), max_slots=4)
    t0 = mcinv.mcinv_pool_submit(pool, c, matrix_id=0, burnin=2, samples=4)
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_pool_submit(pool, c, matrix_id=1, burnin=2, samples=4)
    assert e.value.status == 4
    run_until_done(pool, [t0])
    mcinv.mcinv_pool_release(pool, t0)
    t1 = mcinv.mcinv_pool_submit(pool, c, matrix_id=1, burnin=2, samples=4)
    run_until_done(pool, [t1])
    assert mcinv.mcinv_pool_info(pool)["arena_used"] > 0


def test_pool_batch_estimates_cover_the_dense_inverse():
    sizes = wl.batch_sizes(6, 64, 160, seed=1)
    mats = [wl.random_dominant(int(n), 4, 1.5, 1000 + k) for k, n in enumerate(sizes)]
    # 100 sampling steps, two a batch: 50 batch means, so the z-scores are nearly normal
    pool = mcinv.mcinv_pool_create(K=256, seed=0, mem_budget=1 << 30, max_slots=16, batch_cycles=8, fold_steps=2)
    tickets = [mcinv.mcinv_pool_submit(pool, c, matrix_id=k, burnin=80, samples=800) for k, c in enumerate(mats)]
    run_until_done(pool, tickets)
    zs = []
    for c, t in zip(mats, tickets):
        m, se = mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_BLOCK, c.n)
        truth = np.linalg.inv(c.to_dense())
        zs.append(((m - truth) / se).ravel())
    zs = np.concatenate(zs)
    assert np.mean(np.abs(zs) > 3) < 0.01
    assert 0.8 < np.sqrt(np.mean(zs ** 2)) < 1.25


def test_pool_colour_order_follows_the_oracle_on_the_permuted_matrices():
    """MCINV_F_COLOR_ORDER in a pool: every member samples P C P^T (Sec. 4 reordering),
    so its chains follow the oracle on that matrix, and its diagonal and inverse, mapped
    back to the rows of C, match the oracle's accumulation mapped the same way."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from _greedy import greedy_order, permuted
    K, B, burn, samp = 64, 4, 6, 41  # 11 sampling steps: two folded batches of the default 8 steps
    mats = [wl.random_dominant(n, 4, 1.5, seed) for n, seed in ((90, 4), (333, 5))]
    pool = mcinv.mcinv_pool_create(K=K, seed=13, mem_budget=1 << 28, max_slots=4, batch_cycles=B,
                                   flags=mcinv.MCINV_F_COLOR_ORDER)
    tickets = [mcinv.mcinv_pool_submit(pool, c, matrix_id=7 + k, burnin=burn, samples=samp, want_inverse=True)
               for k, c in enumerate(mats)]
    run_until_done(pool, tickets)
    for k, (c, t) in enumerate(zip(mats, tickets)):
        order, _ = greedy_order(c)
        cp = permuted(c, order)
        z, w, cyc = mcinv.mcinv_pool_get_state(pool, t, c.n)
        st, dacc, _ = oracle.run(cp, K, seed=13, matrix=7 + k, ncycles=burn + samp, acc_from=burn)
        assert rel_err(z[order], st.z.real) < TOL and rel_err(w[order], st.w.real) < TOL
        dm, _ = mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_DIAG, c.n)
        assert rel_err(dm[order], dacc.sum(0).real / (K * samp)) < TOL
        inv, ise = mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_BLOCK, c.n)
        # the whole inverse, entry by entry: the oracle's accumulation on P C P^T (BF16
        # operands, the pool's batches), its rows and columns mapped back to those of C
        import _block_oracle
        F = mcinv.mcinv_pool_info(pool)["fold_steps"]
        om_p, ose_p = _block_oracle.block_estimate(cp, K, 13, 7 + k, burn, samp, B, F)
        om, ose = np.empty_like(om_p), np.empty_like(ose_p)
        om[np.ix_(order, order)] = om_p
        ose[np.ix_(order, order)] = ose_p
        bar = 1e-4 * np.abs(om).max()
        assert np.abs(inv - om).max() <= bar and np.abs(ise - ose).max() <= bar
        q = wl.q_diag(c.n, 2)
        tr, _ = mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_TRACE, c.n, q_diag=q)
        assert abs(tr - (q * dm).sum()) < 1e-9 * abs(tr)
        # the inverse's diagonal is the diagonal estimate, in the rows of C (BF16 products)
        assert np.abs(np.diag(inv) - dm).max() < 2e-2 * np.abs(dm).max()
    mcinv.mcinv_pool_destroy(pool)


@pytest.mark.parametrize("flags,ring_threads,ring_chains", [(0, 384, 128), (mcinv.MCINV_F_COLOR_ORDER, 384, 128),
                                                            (0, 512, 128), (mcinv.MCINV_F_COLOR_ORDER, 512, 128),
                                                            (0, 384, 256), (mcinv.MCINV_F_COLOR_ORDER, 384, 256)])
def test_pool_ring_form_equals_chain_sliced_form(flags, ring_threads, ring_chains):
    # the ring form (a CTA of 12 or 16 warps per 128-chain block, or 12 warps per 256-chain
    # block, bulk-staged gathers) and the chain-sliced form compute the same arithmetic:
    # states and estimates bit for bit (K = 192: a 256-chain block that the chains fill in part)
    K, B, burn, samp = 192, 4, 5, 11
    # 30 entries a row: rows longer than a 24-slot ring run in rounds
    mats = [wl.random_dominant(n, 4, 1.5, 40 + n) for n in (70, 333, 1200)] + [wl.pedigree(900, 1.2, 5),
                                                                                 wl.random_dominant(300, 30, 1.5, 8)]
    res = {}
    for name, shape in (("ring", dict(chains_per_cta=ring_chains, threads_per_cta=ring_threads)),
                        ("sliced", dict(chains_per_cta=32, threads_per_cta=512))):
        pool = mcinv.mcinv_pool_create(K=K, seed=2, mem_budget=1 << 29, max_slots=8, batch_cycles=B, flags=flags,
                                       **shape)
        tickets = [mcinv.mcinv_pool_submit(pool, c, matrix_id=7 + k, burnin=burn, samples=samp, want_inverse=True)
                   for k, c in enumerate(mats)]
        run_until_done(pool, tickets)
        info = mcinv.mcinv_pool_info(pool)
        assert info["chains_per_cta"] == shape["chains_per_cta"] and info["threads_per_cta"] == shape["threads_per_cta"]
        res[name] = [(mcinv.mcinv_pool_get_state(pool, t, c.n),
                      mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_DIAG, c.n),
                      mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_BLOCK, c.n)) for c, t in zip(mats, tickets)]
        mcinv.mcinv_pool_destroy(pool)
    for (sr, dr, br), (ss, ds, bs) in zip(res["ring"], res["sliced"]):
        assert np.array_equal(sr[0], ss[0]) and np.array_equal(sr[1], ss[1]) and sr[2] == ss[2]
        assert np.array_equal(dr[0], ds[0]) and np.array_equal(dr[1], ds[1])
        # (a member whose samples fold as one batch has no batch-means SE: NaN in both)
        assert np.array_equal(br[0], bs[0]) and np.array_equal(br[1], bs[1], equal_nan=True)


@pytest.mark.parametrize("ring_chains", [128, 256])
def test_pool_ring_form_follows_the_oracle(ring_chains):
    K, B, burn, samp = 64, 4, 6, 7
    mats = [wl.random_dominant(n, 4, 1.5, seed) for n, seed in ((64, 1), (517, 3))] + [wl.pedigree(700, 1.2, 2)]
    pool = mcinv.mcinv_pool_create(K=K, seed=11, mem_budget=1 << 28, max_slots=8, batch_cycles=B,
                                   chains_per_cta=ring_chains, threads_per_cta=384)
    tickets = [mcinv.mcinv_pool_submit(pool, c, matrix_id=100 + k, burnin=burn, samples=samp)
               for k, c in enumerate(mats)]
    run_until_done(pool, tickets)
    for k, (c, t) in enumerate(zip(mats, tickets)):
        z, w, cyc = mcinv.mcinv_pool_get_state(pool, t, c.n)
        assert cyc == burn + samp
        st, dacc, _ = oracle.run(c, K, seed=11, matrix=100 + k, ncycles=burn + samp, acc_from=burn)
        assert rel_err(z, st.z.real) < TOL and rel_err(w, st.w.real) < TOL
        dm, _ = mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_DIAG, c.n)
        assert rel_err(dm, dacc.sum(0).real / (K * samp)) < TOL


def test_pool_shape_rejections():
    # chain slices of 4 x a power of two <= 128, or the 256-chain ring form with 384 threads
    for shape in (dict(chains_per_cta=256, threads_per_cta=512), dict(chains_per_cta=96),
                  dict(chains_per_cta=512)):
        with pytest.raises(mcinv.McinvError) as e:
            mcinv.mcinv_pool_create(K=256, seed=1, mem_budget=1 << 26, max_slots=2, **shape)
        assert e.value.status == mcinv.MCINV_E_ARG
    pool = mcinv.mcinv_pool_create(K=256, seed=1, mem_budget=1 << 26, max_slots=2, chains_per_cta=256)
    info = mcinv.mcinv_pool_info(pool)
    assert info["chains_per_cta"] == 256 and info["threads_per_cta"] == 384
    mcinv.mcinv_pool_destroy(pool)


@pytest.mark.parametrize("shape", [dict(chains_per_cta=128, threads_per_cta=384), dict(chains_per_cta=256),
                                   dict(chains_per_cta=32, threads_per_cta=512)])
def test_pool_reports_divergence(shape):
    # C = [[1, 3], [4, 1]]: sp(T) > 1 (Sec. 2.2); the ring form checks the bound on the last
    # cycle of each step, where a diverging chain is still beyond it
    csr = wl.csr_from_coo(2, [0, 0, 1, 1], [0, 1, 0, 1], np.array([1.0, 3.0, 4.0, 1.0]))
    pool = mcinv.mcinv_pool_create(K=64, seed=1, mem_budget=1 << 26, max_slots=2, batch_cycles=8, **shape)
    t = mcinv.mcinv_pool_submit(pool, csr, matrix_id=1, burnin=64, samples=8, want_inverse=False)
    run_until_done(pool, [t])
    with pytest.raises(mcinv.McinvError) as e:
        mcinv.mcinv_pool_estimate(pool, t, mcinv.MCINV_EST_DIAG, csr.n)
    assert e.value.status == mcinv.MCINV_E_DIVERGED
    mcinv.mcinv_pool_destroy(pool)
