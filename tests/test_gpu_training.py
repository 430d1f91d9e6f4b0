"""Differentiation workload: 200 AMSGrad steps of the E + F + W loss (weights 1 / 1 / 0.1)
on the 4-species alloy set at 1000 structures, whole batch per step, FP32 with FP64
reductions.  Checked by the loss falling and, at the final parameters, by the loss and
gradient of a sample of structures against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from _gradcheck import assert_grad_close
from paper_2606_19557_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_200_amsgrad_steps_alloy_1000():
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS["alloy_t4"]
    b = synth.batch_alloy(seed=3, n_struct=1000)
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, 3)
    # normalisation from the descriptors of a sample (an input to both sides)
    qs = oracle.scale_from_range(oracle.descriptors(spec, theta, b.subset(range(40))))
    qs = qs.astype(np.float32).astype(np.float64)
    Er, Fr, Wr = synth.random_targets(b, 7)
    lam = (1.0, 1.0, 0.1)
    nep = NEP(spec)
    nep.set_structures_batch(b)
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    nep.set_targets(Er, Fr, Wr)
    nep.optim_init(lr=2e-3)
    L = []
    l3 = torch.empty(3, dtype=torch.float64, device="cuda")
    for step in range(200):
        nep.train_step(lam, l3)
        if step % 20 == 0 or step == 199:
            L.append(float(np.dot(lam, l3.cpu().numpy())))
    assert np.all(np.isfinite(L))
    assert L[-1] < 0.9 * L[0]
    assert nep.optim_state()["t"] == 200
    th = nep.get_params().cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(th)) and np.max(np.abs(th - theta)) > 1e-3
    # parity at the final parameters on a sample of the batch
    idx = np.arange(0, 1000, 50)
    sub = b.subset(idx)
    a_idx = np.concatenate([np.arange(b.atom_off[i], b.atom_off[i + 1]) for i in idx])
    chk = NEP(spec)
    chk.set_structures_batch(sub)
    chk.set_params(torch.tensor(th, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    l3g, gg = chk.loss_grad(Er[idx], Fr[a_idx], Wr[idx], None, lam)
    l3o, go = oracle.loss_grad(spec, th, qs, sub, Er[idx], Fr[a_idx], Wr[idx], None, lam)[:2]
    np.testing.assert_allclose(l3g.cpu().numpy(), l3o, rtol=1e-5)
    assert_grad_close(gg.cpu().numpy(), go, spec, 1e-5)
