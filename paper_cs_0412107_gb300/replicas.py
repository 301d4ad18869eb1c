"""Replicas on several GPUs: one process per GPU, each with its own handle on its
own range of chains, and the estimates combined at the end.

The chains of the method are independent, and the noise of chain c is keyed by
its global id (``mcinv_options.chain_base`` + local index).  K chains split over
R ranks as contiguous ranges therefore draw exactly what one run with all K
chains draws.  The estimate of the whole run is the chain-weighted mean of the
ranks' estimates (Eq. 1/C averages over chains and cycles), and the ranks'
Monte Carlo errors combine as those of independent estimates.  The data path
needs no exchange; one gather of (estimate, error, weight) per rank at the end
is the only collective.
"""
from __future__ import annotations

import numpy as np


def shard(K_total: int, world: int, rank: int) -> tuple[int, int]:
    """This rank's chains: (count, chain_base).  Contiguous ranges; the first
    K_total % world ranks take one chain more."""
    if world < 1 or not 0 <= rank < world or K_total < world:
        raise ValueError("need 0 <= rank < world <= K_total")
    q, r = divmod(K_total, world)
    count = q + (1 if rank < r else 0)
    base = rank * q + min(rank, r)
    return count, base


def combine(means, ses, weights):
    """The estimate over all ranks from each rank's estimate, standard error and
    weight (chains x samples): the weighted mean, and
    SE^2 = sum_r (w_r / W)^2 SE_r^2 (independent ranks)."""
    w = np.asarray(weights, dtype=np.float64)
    W = w.sum()
    m = np.asarray(means, dtype=np.float64)
    s = np.asarray(ses, dtype=np.float64)
    shape = (-1,) + (1,) * (m.ndim - 1)
    f = (w / W).reshape(shape)
    return (f * m).sum(0), np.sqrt(((f * s) ** 2).sum(0))


def all_gather_combine(mean, se, weight, group=None):
    """Gather every rank's (estimate, SE, weight) with torch.distributed and
    return the combined estimate and SE on every rank.  The arrays travel as
    FP64 tensors on the process group's device (CPU for gloo, the current GPU
    for nccl)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    m = torch.as_tensor(np.ascontiguousarray(mean, dtype=np.float64), device=dev)
    s = torch.as_tensor(np.ascontiguousarray(se, dtype=np.float64), device=dev)
    w = torch.tensor([float(weight)], dtype=torch.float64, device=dev)
    world = dist.get_world_size(group)
    ms = [torch.empty_like(m) for _ in range(world)]
    ss = [torch.empty_like(s) for _ in range(world)]
    ws = [torch.empty_like(w) for _ in range(world)]
    dist.all_gather(ms, m, group=group)
    dist.all_gather(ss, s, group=group)
    dist.all_gather(ws, w, group=group)
    return combine([x.cpu().numpy() for x in ms], [x.cpu().numpy() for x in ss], [float(x.item()) for x in ws])
