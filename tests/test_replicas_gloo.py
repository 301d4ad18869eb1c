"""Replicas across processes (the multi-GPU form, run here as world-size-2 gloo
ranks on the CPU with the oracle as each rank's sampler): the chains split into
disjoint ranges keyed by their global ids reproduce one run with all chains, the
combined estimate equals that run's to rounding, and the bench's cross-rank
helpers (barrier, max over ranks) work over gloo."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_cs_0412107_gb300 import replicas
from paper_cs_0412107_gb300 import workloads as wl

K_TOTAL, BURN, SAMP, SEED = 48, 5, 12, 4


def _matrix():
    return wl.random_dominant(40, 4, 1.5, 3)


def _rank_estimate(K, base, cpg=4):
    # this rank's diagonal estimate and group standard error (groups of cpg chains)
    c = _matrix()
    _, dacc, _ = oracle.run(c, K, seed=SEED, chain0=base, ncycles=BURN + SAMP, acc_from=BURN, cpg=cpg)
    G = dacc.shape[0]
    counts = np.array([min(cpg, K - g * cpg) for g in range(G)], dtype=np.float64)
    mean, se = oracle.group_estimate(dacc, counts, SAMP)
    return mean.real, se.real, K * SAMP


def test_shards_are_disjoint_and_cover_the_chains():
    for K, world in ((48, 2), (50, 3), (7, 7), (1024, 8)):
        got = [replicas.shard(K, world, r) for r in range(world)]
        assert sum(k for k, _ in got) == K
        assert [b for _, b in got] == list(np.cumsum([0] + [k for k, _ in got[:-1]]))
    with pytest.raises(ValueError):
        replicas.shard(3, 4, 0)


def test_split_chains_draw_what_one_run_draws():
    # the state of chains base.. base+K-1 run alone equals those columns of the full run
    c = _matrix()
    full, _, _ = oracle.run(c, K_TOTAL, seed=SEED, ncycles=BURN)
    for r in range(2):
        k, base = replicas.shard(K_TOTAL, 2, r)
        part, _, _ = oracle.run(c, k, seed=SEED, chain0=base, ncycles=BURN)
        assert np.array_equal(part.z, full.z[:, base:base + k]) and np.array_equal(part.w, full.w[:, base:base + k])


def test_combined_mean_equals_one_run():
    c = _matrix()
    _, dacc, _ = oracle.run(c, K_TOTAL, seed=SEED, ncycles=BURN + SAMP, acc_from=BURN)
    ref = dacc.sum(0).real / (K_TOTAL * SAMP)
    parts = [_rank_estimate(*replicas.shard(K_TOTAL, 2, r)) for r in range(2)]
    m, se = replicas.combine([p[0] for p in parts], [p[1] for p in parts], [p[2] for p in parts])
    assert np.abs(m - ref).max() <= 1e-12 * np.abs(ref).max()
    # independent halves: the combined error is about 1/sqrt(2) of one half's
    assert np.all(se > 0) and np.median(se / parts[0][1]) == pytest.approx(2 ** -0.5, rel=0.35)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        k, base = replicas.shard(K_TOTAL, world, rank)
        mean, se, weight = _rank_estimate(k, base)
        m, s = replicas.all_gather_combine(mean, se, weight)
        bench.barrier(world)
        t = bench.max_over_ranks(float(rank + 1), world)
        out.put((rank, m, s, t))
    finally:
        dist.destroy_process_group()


def test_gloo_ranks_combine_to_one_run():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c = _matrix()
    _, dacc, _ = oracle.run(c, K_TOTAL, seed=SEED, ncycles=BURN + SAMP, acc_from=BURN)
    ref = dacc.sum(0).real / (K_TOTAL * SAMP)
    for _, m, s, t in res:
        assert np.abs(m - ref).max() <= 1e-12 * np.abs(ref).max()
        assert t == world  # the max over ranks of rank + 1
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])
