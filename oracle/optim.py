"""FP64 statement of the paper's optimiser and learning-rate schedule.  TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module.  It shares nothing with the CUDA sources.

Follows Sec. "Training" of the paper:
  * Adam with the AMSGrad variant: the biased moments m_t, v_t, their bias-corrected
    forms m^_t = m_t / (1 - beta1^t), v^_t = v_t / (1 - beta2^t), the running maximum
    of the BIAS-CORRECTED second moment v^max_t = max(v^max_{t-1}, v^_t) (this is the
    paper's form; PyTorch's ``amsgrad=True`` keeps the maximum of the raw v_t and
    corrects afterwards, which differs), and the update
    theta_t = theta_{t-1} - eta_t m^_t / (sqrt(v^max_t) + eps);
  * the epoch-level plateau schedule eta_{e+1} = max(gamma eta_e, eta_min), applied
    once the mean loss of an epoch has shown no improvement over p epochs in a row;
  * the two-stage protocol (a stage fixes lambda_E, lambda_F, lambda_V and restarts
    the learning rate; the plateau schedule runs within each stage).

Readings where the paper is silent:
  * parameters are stored in FP32 (the precision of the whole pass); the optimiser's
    moments and arithmetic are FP64, and the new parameters are rounded to FP32 after
    every update;
  * what counts as an improvement: the epoch loss L_e improves iff L_e < best (1 - tau),
    tau >= 0 a relative threshold (0 = any decrease); after p consecutive epochs without
    improvement the rate is reduced and the count restarts;
  * a new stage keeps the Adam moments and the step count, and restarts the schedule
    (learning rate set to the stage's value, best loss forgotten).
"""
from __future__ import annotations

import math

import numpy as np


class AMSGrad:
    """theta (FP32 values held in float64) and the FP64 optimiser state."""

    def __init__(self, theta, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                 store_fp32: bool = True):
        self.store_fp32 = store_fp32
        self.theta = self._store(np.asarray(theta, dtype=np.float64).copy())
        self.beta1, self.beta2, self.eps = float(beta1), float(beta2), float(eps)
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.vmax = np.zeros_like(self.theta)
        self.t = 0

    def _store(self, x):
        return x.astype(np.float32).astype(np.float64) if self.store_fp32 else x

    def step(self, g, lr: float):
        """One update with gradient g at learning rate lr (the moment, bias-correction,
        running-maximum and update equations, in that order)."""
        g = np.asarray(g, dtype=np.float64)
        self.t += 1
        b1, b2 = self.beta1, self.beta2
        self.m = b1 * self.m + (1.0 - b1) * g
        self.v = b2 * self.v + (1.0 - b2) * g * g
        m_hat = self.m / (1.0 - b1 ** self.t)
        v_hat = self.v / (1.0 - b2 ** self.t)
        self.vmax = np.maximum(self.vmax, v_hat)
        self.theta = self._store(self.theta - lr * m_hat / (np.sqrt(self.vmax) + self.eps))
        return self.theta


class Plateau:
    """Epoch-level learning-rate schedule: eta_{e+1} = max(gamma eta_e, eta_min)."""

    def __init__(self, lr: float, factor: float, patience: int, lr_min: float = 0.0, threshold: float = 0.0):
        if not (0.0 < factor < 1.0) or patience < 1:
            raise ValueError("need 0 < factor < 1 and patience >= 1")
        self.lr, self.factor, self.patience = float(lr), float(factor), int(patience)
        self.lr_min, self.threshold = float(lr_min), float(threshold)
        self.best = math.inf
        self.bad = 0
        self.reductions = 0

    def restart(self, lr: float):
        self.lr = float(lr)
        self.best = math.inf
        self.bad = 0

    def epoch_end(self, epoch_loss: float) -> float:
        """Feeds the epoch-averaged loss; returns the rate for the next epoch."""
        if epoch_loss < self.best * (1.0 - self.threshold):
            self.best = float(epoch_loss)
            self.bad = 0
        else:
            self.bad += 1
        if self.bad >= self.patience:
            self.lr = max(self.factor * self.lr, self.lr_min)
            self.bad = 0
            self.reductions += 1
        return self.lr


def two_stage(theta, grad_fn, stages, batches_per_epoch: int, beta1=0.9, beta2=0.999, eps=1e-8, factor=0.5,
              patience=2, lr_min=0.0, threshold=0.0):
    """Runs the two-stage protocol.  ``stages`` = [(epochs, (lamE, lamF, lamV), lr0), ...];
    ``grad_fn(theta, lam, b)`` returns (loss L, gradient) of mini-batch b.  Returns the
    final theta and, per epoch, (stage, learning rate used, epoch-averaged loss)."""
    opt = AMSGrad(theta, beta1, beta2, eps)
    sched = None
    log = []
    for si, (epochs, lam, lr0) in enumerate(stages):
        if sched is None:
            sched = Plateau(lr0, factor, patience, lr_min, threshold)
        else:
            sched.restart(lr0)
        for _ in range(epochs):
            lr = sched.lr
            tot = 0.0
            for b in range(batches_per_epoch):
                L, g = grad_fn(opt.theta, lam, b)
                tot += L
                opt.step(g, lr)
            Le = tot / batches_per_epoch
            log.append((si, lr, Le))
            sched.epoch_end(Le)
    return opt.theta, log
