"""Parity at the full sizes of the benchmark configurations, in the launch configuration the
bench times (autotuned shape).

Structures are independent, so a structure's E_s, F_i and W_s come out of the full batched
pass exactly as from that structure alone: sampled structures are checked one by one
against the FP64 oracle.  The loss and gradient are checked against the oracle on the whole
1000-structure batch (seconds of oracle time).  At the larger sizes the gradient is checked
twice: against the oracle, block by block, through the full-batch adjoint with the
cotangents restricted to a sample of structures (including a 10,000-atom cell), and through
a property that holds at any size: the batch's gradient equals the sum over two shards
evaluated with the batch's normalisers.
"""
import numpy as np
import pytest

import oracle
from _gradcheck import assert_grad_close
from paper_2606_19557_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _setup(name, batch, seed, qs_sample=None):
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS[name]
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, seed)
    src = batch if qs_sample is None else batch.subset(qs_sample)
    qs = oracle.scale_from_range(oracle.descriptors(spec, theta, src)).astype(np.float32).astype(np.float64)
    nep = NEP(spec)
    nep.set_structures_batch(batch)
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    nep.autotune()
    return spec, theta, qs, nep


def _check_sampled_structures(spec, theta, qs, nep, batch, idx):
    E, F, W = [x.cpu().numpy() for x in nep.eval()]
    sub = batch.subset(idx)
    Eo, Fo, Wo = oracle.evaluate(spec, theta, qs, sub)
    a_idx = np.concatenate([np.arange(batch.atom_off[i], batch.atom_off[i + 1]) for i in idx])
    assert rel(E[idx], Eo) < TOL
    assert rel(F[a_idx], Fo) < TOL
    assert rel(W[idx], Wo) < TOL
    cnt = sub.counts()
    assert np.max(np.abs(E[idx] - Eo) / cnt) * 1e3 < 0.1  # meV/atom
    assert np.max(np.abs(F[a_idx] - Fo)) * 1e3 < 1.0       # meV/A


def _subset_backward(spec, theta, qs, nep, batch, idx, seed):
    """The full-batch adjoint (every kernel path the full size reaches: warp ranges spanning
    species runs, per-warp partial slots, the reduction's row groups) with the cotangents
    dE, dF, dW zero outside the structures idx.  Structures are independent, so the result
    is the gradient of those structures alone, which the oracle computes on the subset."""
    rng = np.random.default_rng(seed)
    off = batch.atom_off
    dE = np.zeros(batch.n_struct)
    dF = np.zeros((batch.n_atoms, 3), np.float32)
    dW = np.zeros((batch.n_struct, 9))
    for s in idx:
        dE[s] = rng.normal()
        dF[off[s]:off[s + 1]] = rng.normal(size=(off[s + 1] - off[s], 3)).astype(np.float32)
        dW[s] = rng.normal(size=9)
    nep.eval()
    g = nep.backward(dE, dF, dW).cpu().numpy()
    a_idx = np.concatenate([np.arange(off[s], off[s + 1]) for s in idx])
    go = oracle.backward(spec, theta, qs, batch.subset(idx), dE[idx], dF[a_idx].astype(np.float64), dW[idx])
    assert_grad_close(g, go, spec, TOL)


def _shard_sum_property(spec, theta, qs, nep, batch, Er, Fr, Wr, lam):
    from paper_2606_19557_gb300 import NEP, shard
    l3, g = nep.loss_grad(Er, Fr, Wr, None, lam)
    l3, g = l3.cpu().numpy(), g.cpu().numpy().astype(np.float64)
    norms = shard.global_normalizers(batch.counts())
    L = np.zeros(3)
    G = np.zeros_like(g)
    for idx in shard.partition(batch.counts(), 2):
        sub = batch.subset(idx)
        a_idx = np.concatenate([np.arange(batch.atom_off[i], batch.atom_off[i + 1]) for i in idx])
        part = NEP(spec)
        part.set_structures_batch(sub)
        part.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
        part.set_loss_normalizers(*norms)
        pl, pg = part.loss_grad(Er[idx], Fr[a_idx], Wr[idx], None, lam)
        L += pl.cpu().numpy()
        G += pg.cpu().numpy().astype(np.float64)
        part.close()
    np.testing.assert_allclose(L, l3, rtol=TOL)
    assert rel(G, g) < TOL


def test_bench_workload_1000_structures():
    """The 1000-structure FCC/BCC workload the bench times: sampled E/F/W, and the full
    loss and gradient against the oracle on the whole batch."""
    b = synth.batch_fcc_bcc(seed=2, n_struct=1000)
    spec, theta, qs, nep = _setup("fcc_bcc_t1", b, 1, qs_sample=np.arange(0, 1000, 5))
    rng = np.random.default_rng(0)
    _check_sampled_structures(spec, theta, qs, nep, b, np.sort(rng.choice(1000, 25, replace=False)))
    Er, Fr, Wr = synth.random_targets(b, 3)
    lam = (1.0, 1.0, 0.1)
    l3, g = nep.loss_grad(Er, Fr, Wr, None, lam)
    l3o, go = oracle.loss_grad(spec, theta, qs, b, Er, Fr, Wr, None, lam)[:2]
    np.testing.assert_allclose(l3.cpu().numpy(), l3o, rtol=TOL)
    assert_grad_close(g.cpu().numpy(), go, spec, TOL)


def test_alloy_5000_structures():
    """4-species alloy, 5000 structures of 16-512 atoms with liquid-like and slab structures."""
    b = synth.batch_alloy(seed=3, n_struct=5000)
    spec, theta, qs, nep = _setup("alloy_t4", b, 3, qs_sample=np.arange(0, 5000, 25))
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(5000, 25, replace=False))
    _check_sampled_structures(spec, theta, qs, nep, b, idx)
    _subset_backward(spec, theta, qs, nep, b, idx, 40)
    Er, Fr, Wr = synth.random_targets(b, 4)
    _shard_sum_property(spec, theta, qs, nep, b, Er, Fr, Wr, (1.0, 2.0, 0.3))


def test_scale_20000_structures_and_10000_atom_cells():
    """5 species, 20,000 structures of 2-2000 atoms plus ten 10,000-atom cells, 4- and
    5-body terms, 50 neurons."""
    b = synth.batch_scale(seed=5, n_struct=20000, n_big=10, workers=8)
    spec, theta, qs, nep = _setup("scale_t5", b, 5, qs_sample=np.arange(0, 20000, 100))
    rng = np.random.default_rng(2)
    idx = np.concatenate([np.sort(rng.choice(20000, 20, replace=False)), [20000 + int(rng.integers(10))]])
    _check_sampled_structures(spec, theta, qs, nep, b, idx)
    _subset_backward(spec, theta, qs, nep, b, idx, 50)
    Er, Fr, Wr = synth.random_targets(b, 6)
    _shard_sum_property(spec, theta, qs, nep, b, Er, Fr, Wr, (1.0, 1.0, 0.1))
