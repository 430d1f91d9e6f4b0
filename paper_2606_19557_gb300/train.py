"""Two-stage training protocol (Sec. "Training") driven from the host, computed on the device.

Stage 1 weights forces heavily; stage 2 raises the energy weight and lowers the force
weight and the learning rate.  Within a stage the learning rate follows the epoch-level
plateau schedule.  Every step is ``NEP.train_step`` (loss + gradient + AMSGrad in one
CUDA graph); the host only sequences steps, epoch boundaries and stage starts, and reads
the optimiser state once per epoch for the log.

A new stage keeps the Adam moments and the step count and restarts the schedule at the
stage's learning rate (the paper does not say otherwise).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional, Sequence


@dataclass
class Stage:
    epochs: int
    lam: Sequence[float]  # (lambda_E, lambda_F, lambda_V)
    lr: float


def two_stage(nep, stages: Sequence[Stage], steps_per_epoch: int, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, factor: float = 0.5, patience: int = 5, lr_min: float = 0.0, threshold: float = 0.0,
              step: Optional[Callable] = None) -> list:
    """Runs the stages on ``nep`` (structures, parameters and targets already set).

    ``step(nep, lam, k)`` performs training step k of an epoch; the default is a
    whole-batch ``nep.train_step(lam)``.  Returns one record per epoch: stage, the
    learning rate used in it, and its mean loss."""
    if steps_per_epoch < 1:
        raise ValueError("steps_per_epoch must be >= 1")
    step = step or (lambda n, lam, k: n.train_step(lam))
    log = []
    for si, st in enumerate(stages):
        if si == 0:
            nep.optim_init(st.lr, beta1, beta2, eps, factor, patience, lr_min, threshold)
        else:
            nep.optim_set_lr(st.lr)
        lr = float(st.lr)
        for _ in range(st.epochs):
            for k in range(steps_per_epoch):
                step(nep, st.lam, k)
            nep.optim_epoch_end()
            s = nep.optim_state()  # one host sync per epoch
            log.append({"stage": si, "lr": lr, "loss": s["last_epoch_loss"], "t": s["t"]})
            lr = s["lr"]
    return log
