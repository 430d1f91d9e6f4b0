"""Mini-batch mode: each group of consecutive cached structures against the FP64 oracle
run on that group alone (its own normalisers), through the C ABI."""
import numpy as np
import pytest

import oracle
from _gradcheck import assert_grad_close
from oracle import optim
from paper_2606_19557_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


class MB:
    def __init__(self, name, batch, seed):
        from paper_2606_19557_gb300 import NEP
        self.spec = synth.SPECS[name]
        self.b = batch
        P = oracle.num_params(self.spec)
        self.theta = synth.random_theta(P, seed)
        teacher = synth.random_theta(P, seed + 1)
        self.qs = oracle.scale_from_range(oracle.descriptors(self.spec, self.theta, batch)).astype(np.float32)
        self.qs = self.qs.astype(np.float64)
        E, F, W = oracle.evaluate(self.spec, teacher, self.qs, batch)
        self.E, self.F, self.W = E, F.astype(np.float32).astype(np.float64), W
        self.hw = np.ones(batch.n_struct, np.uint8)
        self.hw[2::5] = 0
        self.nep = NEP(self.spec)
        self.nep.set_structures_batch(batch)
        self.nep.set_params(torch.tensor(self.theta, dtype=torch.float32), torch.tensor(self.qs, dtype=torch.float32))
        self.nep.set_targets(self.E, self.F, self.W, self.hw)

    def oracle_group(self, s0, s1, lam, theta=None):
        idx = np.arange(s0, s1)
        sub = self.b.subset(idx)
        a0, a1 = self.b.atom_off[s0], self.b.atom_off[s1]
        return oracle.loss_grad(self.spec, self.theta if theta is None else theta, self.qs, sub, self.E[idx],
                                self.F[a0:a1], self.W[idx], self.hw[idx], lam)[:2]


_C = {}


def case(name):
    if name not in _C:
        if name == "alloy_t4":
            _C[name] = MB(name, synth.batch_alloy(seed=41, n_struct=14), 41)
        else:
            _C[name] = MB(name, synth.batch_fcc_bcc(seed=42, n_struct=11, n_lo=64, n_hi=128), 42)
    return _C[name]


@pytest.mark.parametrize("name,B", [("alloy_t4", 5), ("alloy_t4", 1), ("fcc_bcc_t1", 4)])
def test_each_group_matches_oracle(name, B):
    c = case(name)
    n = c.nep.minibatch_setup(B)
    assert n == -(-c.b.n_struct // B)
    lam = (1.0, 2.0, 0.3)
    for m in range(n):
        s0, s1 = m * B, min(c.b.n_struct, (m + 1) * B)
        l3, g = c.nep.minibatch_loss_grad(m, lam)
        l3o, go = c.oracle_group(s0, s1, lam)
        np.testing.assert_allclose(l3.cpu().numpy(), l3o, rtol=TOL, atol=1e-300)
        assert_grad_close(g.cpu().numpy(), go, c.spec, TOL)


def test_deterministic_and_reshape():
    c = case("alloy_t4")
    c.nep.minibatch_setup(4)
    a = [c.nep.minibatch_loss_grad(1)[1].cpu().numpy() for _ in range(2)]
    assert np.array_equal(a[0], a[1])
    shape = c.nep.launch_shape()
    c.nep.set_launch(2, 152, 2, 152)  # schedules are rebuilt for the new shape
    g = c.nep.minibatch_loss_grad(1)[1].cpu().numpy()
    c.nep.set_launch(*shape)
    assert rel(g, a[0]) < 1e-6


def test_one_group_is_the_whole_batch():
    c = case("fcc_bcc_t1")
    assert c.nep.minibatch_setup(1000) == 1
    l3m, gm = c.nep.minibatch_loss_grad(0)
    l3, g = c.nep.loss_grad(c.E, c.F, c.W, c.hw)
    np.testing.assert_allclose(l3m.cpu().numpy(), l3.cpu().numpy(), rtol=1e-6)
    assert rel(gm.cpu().numpy(), g.cpu().numpy()) < 1e-6


def test_minibatch_train_step_and_epochs():
    c = case("alloy_t4")
    n = c.nep.minibatch_setup(4)
    c.nep.set_params(torch.tensor(c.theta, dtype=torch.float32), torch.tensor(c.qs, dtype=torch.float32))
    lr = 1e-3
    c.nep.optim_init(lr=lr, factor=0.5, patience=2)
    lam = (1.0, 1.0, 0.1)
    l3 = torch.empty(3, dtype=torch.float64, device="cuda")
    c.nep.minibatch_train_step(2, lam, l3)
    th1 = c.nep.get_params().cpu().numpy().astype(np.float64)
    l3o, go = c.oracle_group(8, 12, lam)
    np.testing.assert_allclose(l3.cpu().numpy(), l3o, rtol=TOL)
    ref = optim.AMSGrad(c.theta)
    ref.step(go, lr)
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    np.testing.assert_allclose((th1 - c.theta)[big], (ref.theta - c.theta)[big], rtol=1e-4, atol=2e-9)
    # epochs driven by the library, shuffled order
    rng = np.random.default_rng(0)
    c.nep.optim_init(lr=5e-3, factor=0.5, patience=2)
    losses = []
    for e in range(12):
        c.nep.minibatch_epoch(rng.permutation(n), lam)
        losses.append(c.nep.optim_state()["last_epoch_loss"])
    st = c.nep.optim_state()
    assert st["t"] == 12 * n
    assert losses[-1] < 0.7 * losses[0]
    # the device parameters agree with the oracle loss at them
    th = c.nep.get_params().cpu().numpy().astype(np.float64)
    l3d = c.nep.minibatch_loss_grad(0, lam)[0].cpu().numpy()
    np.testing.assert_allclose(l3d, c.oracle_group(0, 4, lam, theta=th)[0], rtol=TOL)


def test_padded_copies_follow_updates():
    """A group's pass starts from the padded parameter copies, which every optimiser update
    refreshes in place of a new expansion: after a stand-alone update and a fused training
    step, the pass equals the one after nep_set_params expands the same parameters afresh."""
    c = case("alloy_t4")
    c.nep.minibatch_setup(4)
    qs = torch.tensor(c.qs, dtype=torch.float32)
    c.nep.set_params(torch.tensor(c.theta, dtype=torch.float32), qs)
    c.nep.optim_init(lr=1e-2)
    lam = (1.0, 2.0, 0.3)
    g = np.random.default_rng(7).normal(size=c.nep.P).astype(np.float32)
    c.nep.optim_step(torch.tensor(g))
    c.nep.minibatch_train_step(1, lam)
    th = c.nep.get_params().clone()
    assert not np.array_equal(th.cpu().numpy(), c.theta.astype(np.float32))
    la, ga = c.nep.minibatch_loss_grad(2, lam)
    la, ga = la.cpu().numpy(), ga.cpu().numpy()
    c.nep.set_params(th, qs)
    lb, gb = c.nep.minibatch_loss_grad(2, lam)
    assert np.array_equal(la, lb.cpu().numpy()) and np.array_equal(ga, gb.cpu().numpy())
    c.nep.set_params(torch.tensor(c.theta, dtype=torch.float32), qs)


def test_minibatch_errors():
    from paper_2606_19557_gb300 import NEP, NepError
    spec = synth.SPECS["fcc32_t1"]
    nep = NEP(spec)
    b = synth.batch_fcc32(n_struct=3)
    nep.set_structures_batch(b)
    nep.set_params(torch.zeros(nep.P), torch.ones(nep.n_des))
    with pytest.raises(NepError):
        nep.minibatch_loss_grad(0)  # no setup
    with pytest.raises(NepError):
        nep.minibatch_setup(0)
    assert nep.minibatch_setup(2) == 2
    with pytest.raises(NepError):
        nep.minibatch_loss_grad(0)  # no targets
    E, F, W = np.zeros(3), np.zeros((b.n_atoms, 3)), np.zeros((3, 9))
    nep.set_targets(E, F, W)
    with pytest.raises(NepError):
        nep.minibatch_loss_grad(2)
    nep.optim_init(lr=1e-3)
    with pytest.raises(NepError):
        nep.minibatch_epoch([0, 5])
    nep.set_structures_batch(b)  # invalidates the groups
    with pytest.raises(NepError):
        nep.minibatch_loss_grad(0)
