"""The server: requests admitted into a pool by device memory and run with
continuous batching by an engine thread.

A stream of requests arrives while earlier ones are on the GPU, under a
memory budget too small for all of them at once, so some wait for admission
and the others overlap on the device.  Every result must equal (bit for bit)
the result of the same request served alone, and the latency statistics
must cover every request.
"""
import threading
import time

import numpy as np
import pytest

import _block_oracle
import oracle
from paper_cs_0412107_gb300 import build as libbuild
from paper_cs_0412107_gb300 import mcinv
from paper_cs_0412107_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    libbuild.build()
    mcinv.lib()


KIND = {0: mcinv.MCINV_EST_BLOCK, 1: mcinv.MCINV_EST_DIAG, 2: mcinv.MCINV_EST_TRACE}


def _requests():
    sizes = wl.batch_sizes(10, 64, 600, seed=4)
    out = []
    for k, n in enumerate(sizes):
        c = wl.random_dominant(int(n), 4, 1.5, 500 + k)
        kind = KIND[k % 3]
        q = wl.q_diag(c.n, k) if kind == mcinv.MCINV_EST_TRACE else None
        out.append((c, k, 4 + 3 * k, 20 + 5 * (k % 4), kind, q))
    return out


K, SEED, B, F = 64, 21, 4, 2  # F: sampling steps a block batch (several batches a request)


def _serve(reqs, budget, stagger_s):
    srv = mcinv.mcinv_server_create(K=K, seed=SEED, mem_budget=budget, max_slots=6, batch_cycles=B, fold_steps=F)
    ids = [None] * len(reqs)

    def feed():
        for k, (c, mid, burn, samp, kind, q) in enumerate(reqs):
            ids[k] = mcinv.mcinv_server_submit(srv, c, mid, burn, samp, kind, q)
            time.sleep(stagger_s)

    th = threading.Thread(target=feed)
    th.start()
    th.join()
    results = []
    for k, (c, mid, burn, samp, kind, q) in enumerate(reqs):
        results.append(mcinv.mcinv_server_wait(srv, ids[k], c.n, kind, timeout_s=300))
    stats = mcinv.mcinv_server_stats(srv)
    mcinv.mcinv_server_destroy(srv)
    return results, stats


def test_results_are_the_same_alone_and_in_the_mix():
    reqs = _requests()
    probe = mcinv.mcinv_pool_create(K=64, mem_budget=1 << 24, max_slots=2, batch_cycles=4)
    need = [mcinv.mcinv_pool_footprint(probe, c.n, c.nnz, kind == mcinv.MCINV_EST_BLOCK)
            for c, _, _, _, kind, _ in reqs]
    budget = int(sum(sorted(need)[-3:]) * 1.2)  # room for about three at a time
    mixed, stats = _serve(reqs, budget, 0.002)
    assert stats["completed"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    for k, r in enumerate(reqs):
        alone, _ = _serve([r], max(need[k] * 2, 1 << 24), 0.0)
        m, se, _ = mixed[k]
        m1, se1, _ = alone[0]
        assert np.array_equal(m, m1) and np.array_equal(se, se1, equal_nan=True), k


def test_trace_request_matches_diagonal_request():
    c = wl.random_dominant(300, 4, 1.5, 77)
    q = wl.q_diag(c.n, 3)
    (dres, tres), _ = _serve([(c, 9, 10, 40, mcinv.MCINV_EST_DIAG, None), (c, 9, 10, 40, mcinv.MCINV_EST_TRACE, q)],
                             1 << 28, 0.0)
    assert abs(float(tres[0]) - float((q * dres[0]).sum())) <= 1e-10 * abs(float(tres[0]))


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _oracle_result(c, mid, burn, samp, kind, q, G, F):
    """The FP64 oracle's estimate and SE for one request, from the same draws (the
    request's matrix id keys the noise; chains 0..K-1; cycles counted from 0 at
    admission).  Diagonal and trace: Eq. 1/C and Eq. tr over the sampling cycles,
    SE from the G contiguous chain groups.  Block (the full inverse): the batch
    means of the pool's schedule (B cycles a step, F steps' products a batch), each
    cycle's product formed from the oracle's states rounded to the BF16 operands
    the tensor cores multiply."""
    cpg = K // G
    if kind != mcinv.MCINV_EST_BLOCK:
        _, dacc, _ = oracle.run(c, K, seed=SEED, matrix=mid, ncycles=burn + samp, acc_from=burn, cpg=cpg)
        dacc = dacc.real
        if kind == mcinv.MCINV_EST_TRACE:
            dacc = (dacc * q[None, :]).sum(axis=1)
        return oracle.group_estimate(dacc, np.full(G, cpg), samp)
    return _block_oracle.block_estimate(c, K, SEED, mid, burn, samp, B, F)


def test_served_results_match_the_oracle():
    """Every kind of request (diagonal, trace with q, full inverse), submitted while
    others run under a memory budget for about three at a time: each served estimate
    and standard error equals the FP64 oracle's accumulation of the same draws
    (Eq. 1/C, Eq. tr) within 1e-4 of its largest entry.  The full inverse's SE is held
    to the bar of its mean (1e-4 of the mean's largest entry): BF16 rounding of states
    that sit within FP32 rounding of a BF16 boundary differs between the GPU and the
    oracle, which moves batch means by about 1e-5 of the mean's largest entry, an
    absolute error the much smaller batch-means SE inherits."""
    reqs = _requests()
    probe = mcinv.mcinv_pool_create(K=K, mem_budget=1 << 24, max_slots=2, batch_cycles=B)
    G = mcinv.mcinv_pool_info(probe)["groups"]
    need = [mcinv.mcinv_pool_footprint(probe, c.n, c.nnz, kind == mcinv.MCINV_EST_BLOCK)
            for c, _, _, _, kind, _ in reqs]
    mcinv.mcinv_pool_destroy(probe)
    mixed, stats = _serve(reqs, int(sum(sorted(need)[-3:]) * 1.2), 0.002)
    assert stats["completed"] == len(reqs)
    kinds = set()
    for k, (c, mid, burn, samp, kind, q) in enumerate(reqs):
        m, se, _ = mixed[k]
        om, ose = _oracle_result(c, mid, burn, samp, kind, q, G, F)
        assert _rel(m, om) <= 1e-4, (k, kind, _rel(m, om))
        if kind == mcinv.MCINV_EST_BLOCK:
            assert np.abs(se - ose).max() <= 1e-4 * np.abs(om).max(), (k, kind, _rel(se, om))
        else:
            assert _rel(se, ose) <= 1e-4, (k, kind, _rel(se, ose))
        kinds.add(kind)
    assert kinds == {mcinv.MCINV_EST_BLOCK, mcinv.MCINV_EST_DIAG, mcinv.MCINV_EST_TRACE}
