"""Data-parallel sharding of one loss + gradient pass over structures.

Structures are independent in Eq. "loss": each enters Delta_E, Delta_F and Delta_V
through its own E_s, F_i and W_s, and the three terms are plain sums divided by
batch-wide counts (N_s, N_a, N_s^V).  So a batch can be split into shards, one per
GPU, each shard evaluated with the WHOLE batch's counts as normalisers, and the shards'
loss terms and gradients summed: that sum is the full-batch pass.  The only exchange
is one sum over ranks of [dL/dtheta (P values) | Delta_E, Delta_F, Delta_V] in FP64.

This module holds the host-side parts: the balanced partition, the global
normalisers and the all-reduce.  The per-shard pass itself is ``NEP.loss_grad`` on
the shard, after ``NEP.set_loss_normalizers(*global_normalizers(...))``.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np


def partition(cost: Sequence[float], world: int) -> list:
    """Greedy balance: structures by descending cost, each to the least-loaded rank.

    ``cost`` is one number per structure (atoms x neighbours per atom is a good one;
    the atom count when pairs are not yet known).  Returns ``world`` sorted index
    arrays; ties go to the lowest rank and equal costs keep their input order, so the
    result is the same on every rank.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    c = np.asarray(cost, dtype=np.float64).reshape(-1)
    order = np.argsort(-c, kind="stable")
    load = np.zeros(world)
    parts = [[] for _ in range(world)]
    for s in order:
        r = int(np.argmin(load))
        parts[r].append(int(s))
        load[r] += c[s]
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def global_normalizers(atom_counts: Sequence[int], has_W: Optional[Sequence[int]] = None) -> tuple:
    """(N_s, N_a, N_s^V) of the whole batch: structures, atoms, structures with a virial."""
    n = np.asarray(atom_counts, dtype=np.int64).reshape(-1)
    nsv = n.size if has_W is None else int(np.count_nonzero(np.asarray(has_W).reshape(-1)))
    return float(n.size), float(n.sum()), float(nsv)


def allreduce_loss_grad(loss3, grad, group=None):
    """Sums (loss3 [3], grad [P]) over the ranks of ``group`` in FP64, in place of a copy.

    Returns (loss3, grad) as float64 tensors on the device of ``grad``.  Works with
    any torch.distributed backend; the buffer is a single contiguous FP64 vector so
    the exchange is one collective of (P + 3) x 8 bytes.
    """
    import torch
    import torch.distributed as dist

    g = torch.as_tensor(grad).reshape(-1)
    buf = torch.empty(g.numel() + 3, dtype=torch.float64, device=g.device)
    buf[:g.numel()] = g.to(torch.float64)
    buf[g.numel():] = torch.as_tensor(loss3, dtype=torch.float64, device=g.device).reshape(-1)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf[g.numel():], buf[:g.numel()]
