"""Host-side sequencing of the two-stage protocol (paper_2606_19557_gb300.train), on CPU:
a stand-in context records the calls and keeps its schedule with the oracle's plateau
rule, so the protocol's stage starts, epoch boundaries and log are checked without a GPU."""
import math

import pytest

from oracle import optim
from paper_2606_19557_gb300 import train


class FakeContext:
    def __init__(self, losses):
        self.losses = list(losses)  # mean loss the next epochs report
        self.calls = []
        self.sched = None
        self.t = 0
        self.acc = []
        self.last = math.nan

    def optim_init(self, lr, beta1, beta2, eps, factor, patience, lr_min, threshold):
        self.calls.append(("init", lr))
        self.sched = optim.Plateau(lr, factor, patience, lr_min, threshold)

    def optim_set_lr(self, lr):
        self.calls.append(("set_lr", lr))
        self.sched.restart(lr)

    def train_step(self, lam):
        self.calls.append(("step", tuple(lam)))
        self.t += 1
        self.acc.append(self.losses[0])

    def optim_epoch_end(self):
        self.calls.append(("epoch_end",))
        self.last = sum(self.acc) / len(self.acc)
        self.acc = []
        self.losses.pop(0)
        self.sched.epoch_end(self.last)

    def optim_state(self):
        return {"t": float(self.t), "lr": self.sched.lr, "best": self.sched.best, "bad_epochs": self.sched.bad,
                "last_epoch_loss": self.last, "reductions": self.sched.reductions}


def test_two_stage_sequencing():
    losses = [5.0, 4.0, 4.0, 4.0, 3.0, 2.0, 2.0, 2.0, 2.0]
    ctx = FakeContext(losses)
    stages = [train.Stage(epochs=5, lam=(1.0, 10.0, 0.1), lr=0.1), train.Stage(epochs=4, lam=(10.0, 1.0, 0.1), lr=0.01)]
    log = train.two_stage(ctx, stages, steps_per_epoch=3, factor=0.5, patience=2)
    assert ctx.calls[0] == ("init", 0.1)
    assert ("set_lr", 0.01) in ctx.calls
    assert [r["stage"] for r in log] == [0] * 5 + [1] * 4
    assert [r["loss"] for r in log] == losses
    # stage 1: 5, 4 (better), 4, 4 -> two bad epochs -> 0.05 from epoch 4 on
    assert [r["lr"] for r in log[:5]] == [0.1, 0.1, 0.1, 0.1, 0.05]
    # stage 2 restarts at its own rate: 2 (best), 2, 2 -> two bad epochs -> 0.005 for the last
    assert [r["lr"] for r in log[5:]] == [0.01, 0.01, 0.01, 0.005]
    assert ctx.sched.lr == 0.005
    steps = [c for c in ctx.calls if c[0] == "step"]
    assert len(steps) == 27 and steps[0][1] == (1.0, 10.0, 0.1) and steps[-1][1] == (10.0, 1.0, 0.1)
    assert [r["t"] for r in log] == [3.0 * (k + 1) for k in range(9)]


def test_custom_step_and_validation():
    ctx = FakeContext([1.0, 1.0])
    seen = []
    train.two_stage(ctx, [train.Stage(2, (1.0, 1.0, 0.1), 1e-3)], steps_per_epoch=2,
                    step=lambda n, lam, k: (seen.append(k), n.train_step(lam)))
    assert seen == [0, 1, 0, 1]
    with pytest.raises(ValueError):
        train.two_stage(FakeContext([]), [], steps_per_epoch=0)
