"""Pins of the optimiser oracle (oracle/optim.py) against closed forms and library routines.

CPU only.  Each test targets one plausible mistake:
  * first step and constant gradient: closed forms of the bias-corrected update;
  * gradients of non-decreasing magnitude: the paper's AMSGrad reduces to
    torch.optim.Adam(amsgrad=True) (both maxima are then the current value);
  * decreasing magnitudes: the two variants differ and the oracle keeps the maximum of
    the bias-corrected v^ (catches a port of PyTorch's form);
  * plateau schedule against torch's ReduceLROnPlateau (patience p - 1: torch reduces
    after MORE than `patience` bad epochs) and a hand-worked sequence.
"""
import math

import numpy as np
import pytest

from oracle import optim

torch = pytest.importorskip("torch")


def test_first_step_closed_form():
    rng = np.random.default_rng(0)
    th = rng.normal(size=50)
    g = rng.normal(size=50) * np.logspace(-6, 2, 50)
    o = optim.AMSGrad(th, store_fp32=False)
    lr = 1e-3
    out = o.step(g, lr)
    np.testing.assert_allclose(out, th - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_constant_gradient_closed_form():
    rng = np.random.default_rng(1)
    th = rng.normal(size=20)
    g = rng.normal(size=20)
    o = optim.AMSGrad(th, beta1=0.8, beta2=0.99, eps=1e-6, store_fp32=False)
    lr = 0.01
    for t in range(1, 30):
        o.step(g, lr)
        # m^_t = g and v^_t = g^2 exactly, so every step moves by lr g / (|g| + eps)
        np.testing.assert_allclose(o.theta, th - t * lr * g / (np.abs(g) + 1e-6), rtol=1e-12, atol=1e-14)


def _torch_amsgrad(th, grads, lr, b1=0.9, b2=0.999, eps=1e-8):
    p = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=lr, betas=(b1, b2), eps=eps, amsgrad=True)
    for g in grads:
        opt.zero_grad()
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    return p.detach().numpy()


def test_reduces_to_torch_amsgrad_for_growing_gradients():
    rng = np.random.default_rng(2)
    th = rng.normal(size=40)
    g0 = rng.normal(size=40)
    grads = [g0 * (1.05 ** t) for t in range(25)]  # |g| non-decreasing
    o = optim.AMSGrad(th, store_fp32=False)
    for g in grads:
        o.step(g, 2e-3)
    ref = _torch_amsgrad(th, grads, 2e-3)
    np.testing.assert_allclose(o.theta, ref, rtol=1e-12, atol=1e-14)


def test_max_of_bias_corrected_second_moment():
    rng = np.random.default_rng(3)
    th = rng.normal(size=30)
    g0 = rng.normal(size=30)
    grads = [g0 * (0.7 ** t) for t in range(12)]  # shrinking gradients
    o = optim.AMSGrad(th, store_fp32=False)
    vhats = []
    v = np.zeros(30)
    for t, g in enumerate(grads, start=1):
        o.step(g, 1e-3)
        v = 0.999 * v + 0.001 * g * g
        vhats.append(v / (1 - 0.999 ** t))
        np.testing.assert_allclose(o.vmax, np.max(vhats, axis=0), rtol=1e-13)
    ref = _torch_amsgrad(th, grads, 1e-3)
    # PyTorch keeps max(v_t) and then divides by 1 - beta2^t: a different, smaller denominator
    assert np.max(np.abs(o.theta - ref)) > 1e-6


def test_parameters_are_stored_in_fp32():
    o = optim.AMSGrad(np.array([0.1, -0.2, 0.3]))
    o.step(np.array([1.0, 2.0, -3.0]), 1e-3)
    assert np.array_equal(o.theta, o.theta.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("seed", range(5))
def test_plateau_matches_torch_reduce_on_plateau(seed):
    rng = np.random.default_rng(seed)
    p = int(rng.integers(1, 4))
    factor = float(rng.uniform(0.2, 0.8))
    thr = float(rng.choice([0.0, 1e-4, 1e-2]))
    lr0, lr_min = 0.1, 1e-3
    losses = np.cumsum(rng.normal(-0.05, 0.2, size=60)) + 20.0
    ours = optim.Plateau(lr0, factor, p, lr_min, thr)
    q = torch.tensor([0.0], requires_grad=True)
    opt = torch.optim.SGD([q], lr=lr0)
    ref = torch.optim.lr_scheduler.ReduceLROnPlateau(opt, mode="min", factor=factor, patience=p - 1,
                                                     threshold=thr, threshold_mode="rel", cooldown=0,
                                                     min_lr=lr_min, eps=0.0)
    for L in losses:
        ours.epoch_end(float(L))
        ref.step(float(L))
        assert math.isclose(ours.lr, opt.param_groups[0]["lr"], rel_tol=1e-15)


def test_plateau_hand_sequence():
    s = optim.Plateau(1.0, 0.5, 2, lr_min=0.2)
    seq = [5.0, 4.0, 4.0, 4.5, 3.0, 3.0, 3.0, 3.0, 3.0, 3.0, 3.0]
    # bad epochs: 4.0 (1), 4.5 (2 -> reduce to 0.5), 3.0 improves, then 3.0 x2 -> 0.25,
    # x2 -> 0.2 (floor), x2 -> 0.2
    lrs = [s.epoch_end(x) for x in seq]
    assert lrs == [1.0, 1.0, 1.0, 0.5, 0.5, 0.5, 0.25, 0.25, 0.2, 0.2, 0.2]
    assert s.reductions == 4
    s.restart(0.05)
    assert s.lr == 0.05 and s.best == math.inf and s.bad == 0
    with pytest.raises(ValueError):
        optim.Plateau(1.0, 1.0, 2)
    with pytest.raises(ValueError):
        optim.Plateau(1.0, 0.5, 0)


def test_two_stage_on_a_quadratic():
    """Stage 2 restarts the rate and switches the loss weights; the schedule only ever
    lowers the rate within a stage."""
    target = np.array([1.0, -2.0, 0.5])

    def grad_fn(th, lam, b):
        w = np.array(lam)
        r = th - target
        return float(np.sum(w * r * r)), 2.0 * w * r

    th, log = optim.two_stage(np.zeros(3), grad_fn, [(30, (1.0, 4.0, 0.1), 0.05), (20, (4.0, 1.0, 0.1), 0.01)],
                              batches_per_epoch=4, factor=0.5, patience=2)
    assert len(log) == 50
    st1 = [r for r in log if r[0] == 0]
    st2 = [r for r in log if r[0] == 1]
    assert all(a[1] >= b[1] for a, b in zip(st1, st1[1:]))
    assert st2[0][1] == 0.01
    assert log[-1][2] < log[0][2] * 1e-2
