"""Device optimiser (AMSGrad with the maximum of the bias-corrected second moment, plateau
schedule, training step) against the FP64 optimiser oracle, through the C ABI.

Gradients and epoch losses fed to both sides are seeded test inputs (never GPU results).
Parameters are FP32 on both sides; moments are FP64 on both sides, so the two agree to
within one FP32 rounding of theta per step (the bias corrections are computed as running
products on the device and as powers in the oracle).
"""
import numpy as np
import pytest

import oracle
from oracle import optim
from paper_2606_19557_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ulps(a, b):
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    return np.abs(a.astype(np.float64) - b.astype(np.float64)) / np.spacing(np.maximum(np.abs(a), np.abs(b)))


def _nep(name="fcc32_t1", batch=None):
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS[name]
    b = batch if batch is not None else synth.batch_fcc32(n_struct=2)
    nep = NEP(spec)
    nep.set_structures_batch(b)
    return spec, b, nep


def test_amsgrad_steps_match_oracle():
    spec, b, nep = _nep()
    P = nep.P
    theta0 = synth.random_theta(P, 5)
    nep.set_params(torch.tensor(theta0, dtype=torch.float32), torch.ones(nep.n_des))
    cfg = dict(beta1=0.85, beta2=0.99, eps=1e-7)
    nep.optim_init(lr=3e-3, factor=0.5, patience=2, **cfg)
    ref = optim.AMSGrad(theta0, **cfg)
    rng = np.random.default_rng(11)
    scale = np.logspace(-4, 1, P)
    for t in range(15):
        # growing then shrinking magnitudes, so that both branches of the running maximum occur
        mag = 1.3 ** t if t < 8 else 1.3 ** 8 * 0.5 ** (t - 8)
        g = (rng.normal(size=P) * scale * mag).astype(np.float32)
        g[::17] = 0.0
        nep.optim_step(torch.tensor(g))
        ref.step(g.astype(np.float64), 3e-3)
        th = nep.get_params().cpu().numpy()
        assert np.max(_ulps(th, ref.theta)) <= 1.0, t
    st = nep.optim_state()
    assert st["t"] == 15 and st["lr"] == 3e-3 and np.isnan(st["last_epoch_loss"])


def test_plateau_schedule_matches_oracle():
    spec, b, nep = _nep()
    nep.set_params(torch.zeros(nep.P), torch.ones(nep.n_des))
    nep.optim_init(lr=0.2, factor=0.3, patience=3, lr_min=1e-3, threshold=1e-3)
    ref = optim.Plateau(0.2, 0.3, 3, 1e-3, 1e-3)
    rng = np.random.default_rng(4)
    zero = torch.zeros(nep.P, dtype=torch.float32)
    epochs = np.cumsum(rng.normal(-0.02, 0.1, size=(40, 3)), axis=0) + 5.0
    for e, losses in enumerate(epochs):
        for L in losses:
            nep.optim_step(zero, torch.tensor([L], dtype=torch.float64))
        nep.optim_epoch_end()
        ref.epoch_end(float(np.mean(losses)))
        st = nep.optim_state()
        assert st["lr"] == pytest.approx(ref.lr, rel=1e-15), e
        assert st["bad_epochs"] == ref.bad and st["reductions"] == ref.reductions
        assert st["last_epoch_loss"] == pytest.approx(float(np.mean(losses)), rel=1e-15)
    assert ref.reductions >= 1
    # zero gradients leave the parameters untouched
    assert np.all(nep.get_params().cpu().numpy() == 0.0)
    # a stage restart sets the rate and forgets the best loss
    nep.optim_set_lr(0.05)
    st = nep.optim_state()
    assert st["lr"] == 0.05 and st["best"] == float("inf") and st["bad_epochs"] == 0


def test_train_step_matches_oracle_first_step():
    spec = synth.SPECS["alloy_t4"]
    b = synth.batch_alloy(seed=23, n_struct=6)
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, 23)
    teacher = synth.random_theta(P, 24)
    qs = oracle.scale_from_range(oracle.descriptors(spec, theta, b)).astype(np.float32).astype(np.float64)
    E, F, W = oracle.evaluate(spec, teacher, qs, b)
    F = F.astype(np.float32).astype(np.float64)
    lam = (1.0, 2.0, 0.3)
    from paper_2606_19557_gb300 import NEP
    nep = NEP(spec)
    nep.set_structures_batch(b)
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    nep.set_targets(E, F, W)
    lr = 1e-3
    nep.optim_init(lr=lr)
    l3 = nep.train_step(lam).cpu().numpy()
    th1 = nep.get_params().cpu().numpy().astype(np.float64)
    l3o, go = oracle.loss_grad(spec, theta, qs, b, E, F, W, None, lam)[:2]
    np.testing.assert_allclose(l3, l3o, rtol=1e-5)
    ref = optim.AMSGrad(theta)
    ref.step(go, lr)
    # first step: theta moves by lr g/(|g| + eps); compare where the sign of g is well defined
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    np.testing.assert_allclose((th1 - theta)[big], (ref.theta - theta)[big], rtol=1e-4, atol=2e-9)
    # |step| <= lr, up to the FP32 rounding of the stored parameter
    assert np.all(np.abs(th1 - theta) <= lr * (1 + 1e-6) + np.spacing(np.float32(np.abs(theta) + lr)))
    st = nep.optim_state()
    assert st["t"] == 1
    # the epoch mean of one step is that step's weighted loss
    nep.optim_epoch_end()
    assert nep.optim_state()["last_epoch_loss"] == pytest.approx(float(np.dot(lam, l3o)), rel=1e-5)


def test_two_stage_training_lowers_the_loss():
    """Whole-batch training on device through the two-stage protocol (stage 1 force-heavy,
    stage 2 energy-heavy at a lower rate): the loss falls and the schedule behaves."""
    from paper_2606_19557_gb300 import train
    spec = synth.SPECS["fcc_bcc_t1"]
    b = synth.batch_fcc_bcc(seed=31, n_struct=16, n_lo=64, n_hi=96)
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, 31)
    teacher = synth.random_theta(P, 32)
    qs = oracle.scale_from_range(oracle.descriptors(spec, theta, b)).astype(np.float32).astype(np.float64)
    E, F, W = oracle.evaluate(spec, teacher, qs, b)
    from paper_2606_19557_gb300 import NEP
    nep = NEP(spec)
    nep.set_structures_batch(b)
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    nep.set_targets(E, F.astype(np.float32), W)
    stages = [train.Stage(epochs=30, lam=(1.0, 10.0, 0.1), lr=2e-2), train.Stage(epochs=20, lam=(10.0, 1.0, 0.1), lr=5e-3)]
    log = train.two_stage(nep, stages, steps_per_epoch=4, factor=0.5, patience=3)
    assert len(log) == 50
    s1 = [r for r in log if r["stage"] == 0]
    s2 = [r for r in log if r["stage"] == 1]
    assert s1[-1]["loss"] < 0.5 * s1[0]["loss"]
    assert all(x["lr"] >= y["lr"] for x, y in zip(s1, s1[1:]))
    assert s2[0]["lr"] == 5e-3
    for r in log:
        k = np.log(r["lr"] / (2e-2 if r["stage"] == 0 else 5e-3)) / np.log(0.5)
        assert abs(k - round(k)) < 1e-9
    # the device parameters changed and the loss at them matches the oracle there
    th = nep.get_params().cpu().numpy().astype(np.float64)
    l3 = nep.loss_grad(E, F.astype(np.float32), W, None, (1.0, 1.0, 0.1))[0].cpu().numpy()
    l3o = oracle.loss_grad(spec, th, qs, b, E, F.astype(np.float32), W, None, (1.0, 1.0, 0.1))[0]
    np.testing.assert_allclose(l3, l3o, rtol=1e-5)


def test_optimizer_errors():
    from paper_2606_19557_gb300 import NepError
    spec, b, nep = _nep()
    with pytest.raises(NepError):
        nep.optim_step(torch.zeros(nep.P))  # no optimiser yet
    with pytest.raises(NepError):
        nep.optim_init(lr=-1.0)
    with pytest.raises(NepError):
        nep.optim_init(lr=1e-3, factor=1.5)
    with pytest.raises(NepError):
        nep.optim_init(lr=1e-3, patience=0)
    nep.set_params(torch.zeros(nep.P), torch.ones(nep.n_des))
    nep.optim_init(lr=1e-3)
    with pytest.raises(NepError):
        nep.train_step()  # no targets
    with pytest.raises(NepError):
        nep.optim_set_lr(0.0)
