"""Data-parallel sharding on CPU: two gloo ranks, each running the FP64 oracle on its
shard with the whole batch's normalisers, then one FP64 all-reduce.  The sum must be
the full-batch loss and gradient of Eq. "loss" (structures enter it independently,
so only rounding order differs).
"""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
from paper_2606_19557_gb300 import shard, synth

LAM = (1.0, 2.0, 0.3)


def _case():
    s = synth.SPECS["alloy_t4"]
    b = synth.batch_alloy(seed=31, n_struct=5, n_types=s.n_types, n_lo=6, n_hi=14)
    theta = synth.random_theta(oracle.num_params(s), 31)
    qs = oracle.scale_from_range(oracle.descriptors(s, theta, b))
    Er, Fr, Wr = synth.random_targets(b, 32)
    has_W = np.array([1, 0, 1, 1, 0], np.uint8)
    return s, b, theta, qs, Er, Fr, Wr, has_W


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, b, theta, qs, Er, Fr, Wr, has_W = _case()
        parts = shard.partition(b.counts(), world)
        idx = parts[rank]
        sub = b.subset(idx)
        a_idx = np.concatenate([np.arange(b.atom_off[i], b.atom_off[i + 1]) for i in idx])
        norms = shard.global_normalizers(b.counts(), has_W)
        loss3, g = oracle.loss_grad(s, theta, qs, sub, Er[idx], Fr[a_idx], Wr[idx], has_W[idx], LAM,
                                    norms=np.array(norms))[:2]
        L, G = shard.allreduce_loss_grad(torch.from_numpy(loss3), torch.from_numpy(g))
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([L.numpy(), G.numpy()]))
    finally:
        dist.destroy_process_group()


def test_partition_covers_and_balances():
    rng = np.random.default_rng(0)
    cost = rng.integers(16, 512, size=101).astype(float)
    for world in (1, 2, 3, 8):
        parts = shard.partition(cost, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(cost.size))
        loads = np.array([cost[p].sum() for p in parts])
        # greedy LPT: the spread is at most the largest single item
        assert loads.max() - loads.min() <= cost.max()
        # deterministic
        again = shard.partition(cost, world)
        assert all(np.array_equal(a, c) for a, c in zip(parts, again))
    assert [p.tolist() for p in shard.partition([5, 5], 3)] == [[0], [1], []]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


def test_global_normalizers():
    assert shard.global_normalizers([3, 4, 5]) == (3.0, 12.0, 3.0)
    assert shard.global_normalizers([3, 4, 5], [1, 0, 1]) == (3.0, 12.0, 2.0)
    assert shard.global_normalizers([3, 4], [0, 0]) == (2.0, 7.0, 0.0)


def test_shards_sum_to_full_batch_gloo():
    import torch.multiprocessing as mp
    s, b, theta, qs, Er, Fr, Wr, has_W = _case()
    loss_full, g_full = oracle.loss_grad(s, theta, qs, b, Er, Fr, Wr, has_W, LAM)[:2]
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank, args=(world, _free_port(), d), nprocs=world, start_method="spawn", join=True)
        res = [np.load(os.path.join(d, f"r{r}.npy")) for r in range(world)]
    # every rank holds the same reduced vector
    assert np.array_equal(res[0], res[1])
    L, G = res[0][:3], res[0][3:]
    np.testing.assert_allclose(L, loss_full, rtol=1e-12, atol=0)
    assert np.linalg.norm(G - g_full) <= 1e-12 * np.linalg.norm(g_full)
