"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerance (FP32 path): norm-wise relative error ||x - x_oracle|| / ||x_oracle|| <= 1e-5
on E, F, W, the loss terms and the parameter gradient.  Neighbour lists are compared
bit-exactly (the inclusion decision is an integer taken in float in both).
Inputs are seeded synthetic structures; references come from the oracle's teacher
model, never from the GPU.
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
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def f32(x):
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


class Case:
    """Batch + student/teacher parameters + oracle references (all float32-representable)."""

    def __init__(self, name, batch, seed=1):
        from paper_2606_19557_gb300 import NEP
        self.spec = synth.SPECS[name]
        self.batch = batch
        P = oracle.num_params(self.spec)
        self.theta = synth.random_theta(P, seed)
        self.teacher = synth.random_theta(P, seed + 1)
        q = oracle.descriptors(self.spec, self.theta, batch)
        self.qs = f32(oracle.scale_from_range(q))
        E_t, F_t, W_t = oracle.evaluate(self.spec, self.teacher, self.qs, batch)
        self.E_ref, self.F_ref, self.W_ref = E_t, f32(F_t), W_t
        self.nep = NEP(self.spec)
        self.nep.set_structures_batch(batch)
        self.nep.set_params(torch.tensor(self.theta, dtype=torch.float32), torch.tensor(self.qs, dtype=torch.float32))


def small_cases():
    return {
        "fcc32_t1": lambda: synth.batch_fcc32(),
        "fcc_bcc_t1": lambda: synth.batch_fcc_bcc(seed=12, n_struct=24),
        "alloy_t4": lambda: synth.batch_alloy(seed=13, n_struct=14),
        "scale_t5": lambda: synth.batch_scale(seed=14, n_struct=40, n_big=0),
        "carbon_table1": lambda: synth.batch_fcc_bcc(seed=15, n_struct=4, n_lo=40, n_hi=90),
    }


_CACHE = {}


def get_case(name):
    if name not in _CACHE:
        _CACHE[name] = Case(name, small_cases()[name]())
    return _CACHE[name]


NAMES = list(small_cases().keys())


# ----------------------------------------------------------------------------- neighbours

def _gpu_pairs(nep):
    off, j, s, a = nep.neighbors()
    off = off.cpu().numpy()
    i = np.repeat(np.arange(len(off) - 1), np.diff(off))
    return i, j.cpu().numpy().astype(np.int64), s.cpu().numpy(), a.cpu().numpy().astype(bool), off


def _check_neighbors(nep, batch, rc_R, rc_A):
    gi, gj, gs, ga, off = _gpu_pairs(nep)
    oi, oj, os_, oa = oracle.neighbors(batch, rc_R, rc_A)
    g = set(zip(gi.tolist(), gj.tolist(), map(tuple, gs.tolist()), ga.tolist()))
    o = set(zip(oi.tolist(), oj.tolist(), map(tuple, os_.tolist()), oa.tolist()))
    assert len(g) == len(gi), "duplicate neighbour entries"
    assert g == o
    # angular neighbours first, each group sorted by (species of j, j, S)
    types = np.asarray(batch.types)
    for k in range(min(len(off) - 1, 300)):
        sl = slice(off[k], off[k + 1])
        ang = ga[sl]
        assert np.all(np.diff(ang.astype(int)) <= 0)
        for grp in (True, False):
            m = ang == grp
            key = list(zip(types[gj[sl][m]].tolist(), gj[sl][m].tolist(), map(tuple, gs[sl][m].tolist())))
            assert key == sorted(key)


@pytest.mark.parametrize("name", NAMES)
def test_neighbor_lists_bit_exact(name):
    c = get_case(name)
    _check_neighbors(c.nep, c.batch, c.spec.rc_R, c.spec.rc_A)
    nr, na = c.nep.num_pairs()
    i, j, S, ang = oracle.neighbors(c.batch, c.spec.rc_R, c.spec.rc_A)
    assert nr == len(i) and na == int(ang.sum())


def test_neighbor_edge_geometries():
    """Primitive triclinic cell (self images), a lone atom, a dimer, atoms far outside
    their cell (unwrapped), and a thin cell needing many images."""
    from paper_2606_19557_gb300 import NEP
    a = 3.6
    prim = 0.5 * a * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], float)
    rng = np.random.default_rng(0)
    thin = np.diag([2.0, 2.3, 30.0]) + 0.1 * rng.normal(size=(3, 3))
    structs = [
        (np.array([[0.1, 0.2, 0.3]]), prim),
        (np.array([[5.0, 5.0, 5.0]]), np.eye(3) * 20.0),
        (np.array([[6.0, 6.0, 6.0], [7.9, 6.5, 6.2]]), np.eye(3) * 12.0),
        (rng.uniform(0, 8, size=(10, 3)) + np.array([30.0, -41.0, 17.0]), np.eye(3) * 8.0 + 0.2 * np.eye(3)[::-1]),
        (rng.uniform(0, 1, size=(3, 3)) @ thin, thin),
    ]
    off = np.cumsum([0] + [p.shape[0] for p, _ in structs])
    batch = synth.Batch(off.astype(np.int64), np.concatenate([p for p, _ in structs]).astype(np.float32),
                        np.zeros(off[-1], np.int32), np.stack([c.reshape(9) for _, c in structs]).astype(np.float32), 1)
    spec = synth.SPECS["fcc_bcc_t1"]
    nep = NEP(spec)
    nep.set_structures_batch(batch)
    _check_neighbors(nep, batch, 6.0, 4.0)
    # the degenerate environments (no neighbour at all, one neighbour, self images only)
    # through the whole pass
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, 70)
    qs = f32(oracle.scale_from_range(oracle.descriptors(spec, theta, batch)))
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    E, F, W = [x.cpu().numpy() for x in nep.eval()]
    Eo, Fo, Wo = oracle.evaluate(spec, theta, qs, batch)
    assert rel(E, Eo) < TOL and rel(F, Fo) < TOL and rel(W, Wo) < TOL
    Er, Fr, Wr = synth.random_targets(batch, 71)
    l3, g = nep.loss_grad(Er, Fr, Wr, None, (1.0, 2.0, 0.3))
    l3o, go = oracle.loss_grad(spec, theta, qs, batch, Er, Fr, Wr, None, (1.0, 2.0, 0.3))[:2]
    np.testing.assert_allclose(l3.cpu().numpy(), l3o, rtol=TOL)
    assert_grad_close(g.cpu().numpy(), go, spec, TOL)


# ----------------------------------------------------------------------------- forward


def test_neighbor_dense_cells():
    """Compressed FCC cells (a = 3.5 ... 2.2 A; about 85 to 340 radial neighbours per atom):
    lists longer than the per-atom key scratch (second scan), the staged sort at up to 8
    keys per lane and the unstaged sort beyond 256 keys, bit-exact against brute force;
    E/F/W against the oracle."""
    from paper_2606_19557_gb300 import NEP
    rng = np.random.default_rng(5)
    basis = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], float)
    grid = np.array([[x, y, z] for x in range(3) for y in range(3) for z in range(3)], float)
    frac = (grid[:, None, :] + basis[None, :, :]).reshape(-1, 3) / 3.0
    structs = []
    for a in (3.5, 3.1, 2.8, 2.5, 2.2):
        cell = np.eye(3) * 3 * a
        structs.append((frac @ cell + rng.normal(scale=0.05, size=frac.shape), cell))
    off = np.cumsum([0] + [p.shape[0] for p, _ in structs])
    batch = synth.Batch(off.astype(np.int64), np.concatenate([p for p, _ in structs]).astype(np.float32),
                        rng.integers(0, 2, size=off[-1]).astype(np.int32),
                        np.stack([c.reshape(9) for _, c in structs]).astype(np.float32), 2)
    spec = synth.SPECS["alloy_t4"]
    spec = synth.ModelSpec(2, spec.rc_R, spec.rc_A, 4, 4, 8, 8, 4, 1, 0, 16)
    nep = NEP(spec)
    nep.set_structures_batch(batch)
    _check_neighbors(nep, batch, spec.rc_R, spec.rc_A)
    counts = np.diff(nep.neighbors()[0].cpu().numpy())
    assert counts.min() < 128 and counts.max() > 256
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, 6)
    qs = f32(oracle.scale_from_range(oracle.descriptors(spec, theta, batch)))
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    E, F, W = [x.cpu().numpy() for x in nep.eval()]
    Eo, Fo, Wo = oracle.evaluate(spec, theta, qs, batch)
    assert rel(E, Eo) < TOL and rel(F, Fo) < TOL and rel(W, Wo) < TOL
    nep.close()

@pytest.mark.parametrize("name", NAMES)
def test_descriptors(name):
    c = get_case(name)
    q = c.nep.descriptors().cpu().numpy()
    qo = oracle.descriptors(c.spec, c.theta, c.batch)
    for v in range(qo.shape[1]):
        assert rel(q[:, v], qo[:, v]) < TOL, v


@pytest.mark.parametrize("name", NAMES)
def test_energy_force_virial(name):
    c = get_case(name)
    E, F, W = [x.cpu().numpy() for x in c.nep.eval()]
    Eo, Fo, Wo = oracle.evaluate(c.spec, c.theta, c.qs, c.batch)
    assert rel(E, Eo) < TOL
    assert rel(F, Fo) < TOL
    assert rel(W, Wo) < TOL
    # per-atom view (meV/atom, meV/A) for the report
    cnt = c.batch.counts()
    assert np.max(np.abs(E - Eo) / cnt) * 1e3 < 0.1
    assert np.max(np.abs(F - Fo)) * 1e3 < 1.0


@pytest.mark.parametrize("name", NAMES)
def test_loss_and_gradient(name):
    c = get_case(name)
    hw = np.ones(c.batch.n_struct, np.uint8)
    hw[::3] = 0
    lam = (1.0, 2.0, 0.3)
    l3, g = c.nep.loss_grad(c.E_ref, c.F_ref, c.W_ref, hw, lam)
    l3, g = l3.cpu().numpy(), g.cpu().numpy()
    l3o, go = oracle.loss_grad(c.spec, c.theta, c.qs, c.batch, c.E_ref, c.F_ref, c.W_ref, hw, lam)[:2]
    np.testing.assert_allclose(l3, l3o, rtol=TOL)
    assert_grad_close(g, go, c.spec, TOL)


@pytest.mark.parametrize("name", ["fcc_bcc_t1", "alloy_t4", "scale_t5"])
def test_backward_vjp(name):
    c = get_case(name)
    rng = np.random.default_rng(5)
    dE = rng.normal(size=c.batch.n_struct)
    dF = f32(rng.normal(size=(c.batch.n_atoms, 3)))
    dW = rng.normal(size=(c.batch.n_struct, 9))
    c.nep.eval()
    g = c.nep.backward(dE, dF, dW).cpu().numpy()
    go = oracle.backward(c.spec, c.theta, c.qs, c.batch, dE, dF, dW)
    assert_grad_close(g, go, c.spec, TOL)


def test_autograd_function_matches_oracle():
    from paper_2606_19557_gb300 import NEPFunction
    c = get_case("alloy_t4")
    th = torch.tensor(c.theta, dtype=torch.float32, device="cuda", requires_grad=True)
    E, F, W = NEPFunction.apply(th, c.nep)
    cnt = torch.tensor(c.batch.counts(), dtype=torch.float64, device="cuda")
    Er = torch.tensor(c.E_ref, device="cuda")
    Fr = torch.tensor(c.F_ref, dtype=torch.float32, device="cuda")
    Wr = torch.tensor(c.W_ref, device="cuda")
    L = (((E - Er) / cnt) ** 2).mean() + ((F - Fr) ** 2).double().sum() / (3 * F.shape[0]) \
        + 0.1 * (((W - Wr) / cnt[:, None]) ** 2).sum() / (9 * W.shape[0])
    L.backward()
    go = oracle.loss_grad(c.spec, c.theta, c.qs, c.batch, c.E_ref, c.F_ref, c.W_ref, None, (1.0, 1.0, 0.1))[1]
    assert_grad_close(th.grad.cpu().numpy(), go, c.spec, TOL)


# ----------------------------------------------------------------------------- properties

def test_deterministic_and_graph_replay():
    c = get_case("alloy_t4")
    out = [c.nep.loss_grad(c.E_ref, c.F_ref, c.W_ref) for _ in range(3)]
    g0 = out[0][1].cpu().numpy()
    for l3, g in out[1:]:
        assert np.array_equal(g.cpu().numpy(), g0)
        assert np.array_equal(l3.cpu().numpy(), out[0][0].cpu().numpy())


def test_teacher_gives_near_zero_loss():
    c = get_case("fcc_bcc_t1")
    E, F, W = oracle.evaluate(c.spec, c.theta, c.qs, c.batch)
    l3, g = c.nep.loss_grad(E, f32(F), W)
    l3 = l3.cpu().numpy()
    # references are the student's own FP64 values: residuals are FP32 rounding only
    assert l3[0] < 1e-10 and l3[1] < 1e-10 and l3[2] < 1e-10


def test_host_entry_point_matches_device_call():
    c = get_case("fcc_bcc_t1")
    c.nep.set_targets(c.E_ref, c.F_ref, c.W_ref)
    l3h, gh = c.nep.loss_grad_host(torch.tensor(c.theta, dtype=torch.float32), (1.0, 1.0, 0.1))
    l3d, gd = c.nep.loss_grad(c.E_ref, c.F_ref, c.W_ref, None, (1.0, 1.0, 0.1))
    assert np.array_equal(gh.numpy(), gd.cpu().numpy())
    assert np.array_equal(l3h.numpy(), l3d.cpu().numpy())


def test_launch_shapes_agree():
    c = get_case("scale_t5")
    g0 = c.nep.loss_grad(c.E_ref, c.F_ref, c.W_ref)[1].cpu().numpy()
    shape = c.nep.launch_shape()
    c.nep.set_launch(2, 152, 4, 152 * 2)
    g1 = c.nep.loss_grad(c.E_ref, c.F_ref, c.W_ref)[1].cpu().numpy()
    from paper_2606_19557_gb300 import NepError
    with pytest.raises(NepError):  # blocks hold at most 4 warps
        c.nep.set_launch(8, 152, 4, 152)
    c.nep.set_launch(*shape)
    assert rel(g1, g0) < 1e-6


@pytest.mark.parametrize("name", ["alloy_t4", "scale_t5"])
def test_every_kernel_variant_matches_oracle(name):
    """Each kernel variant (8, 16 or 32 lanes per atom; 128 or 96 registers), forward and
    adjoint alike, against the oracle: E/F/W, the loss and the gradient block by block."""
    c = get_case(name)
    lam = (1.0, 2.0, 0.3)
    Eo, Fo, Wo = oracle.evaluate(c.spec, c.theta, c.qs, c.batch)
    l3o, go = oracle.loss_grad(c.spec, c.theta, c.qs, c.batch, c.E_ref, c.F_ref, c.W_ref, None, lam)[:2]
    shape, var = c.nep.launch_shape(), c.nep.variant()
    lanes = []
    for v in range(6):
        c.nep.set_variant(v, v)
        lanes.append(c.nep.variant()[0])
        E, F, W = [x.cpu().numpy() for x in c.nep.eval()]
        assert rel(E, Eo) < TOL and rel(F, Fo) < TOL and rel(W, Wo) < TOL, v
        l3, g = c.nep.loss_grad(c.E_ref, c.F_ref, c.W_ref, None, lam)
        np.testing.assert_allclose(l3.cpu().numpy(), l3o, rtol=TOL)
        assert_grad_close(g.cpu().numpy(), go, c.spec, TOL)
    assert lanes == [8, 8, 16, 16, 32, 32]
    # back to the earlier variants and shape for the other tests

    def index(lanes, regs):
        return {8: 0, 16: 2, 32: 4}[lanes] + (1 if regs == 96 else 0)

    c.nep.set_variant(index(var[0], var[1]), index(var[2], var[3]))
    c.nep.set_launch(*shape)


def test_empty_batch():
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS["fcc32_t1"]
    nep = NEP(spec)
    empty = synth.Batch(np.zeros(1, np.int64), np.zeros((0, 3), np.float32), np.zeros(0, np.int32),
                        np.zeros((0, 9), np.float32), 1)
    nep.set_structures_batch(empty)
    P = oracle.num_params(spec)
    nep.set_params(torch.zeros(P), torch.ones(nep.n_des))
    E, F, W = nep.eval()
    assert E.numel() == 0 and F.numel() == 0
    l3, g = nep.loss_grad(np.zeros(0), np.zeros((0, 3)), np.zeros((0, 9)))
    assert np.all(l3.cpu().numpy() == 0) and np.all(g.cpu().numpy() == 0)


def test_invalid_inputs_return_errors():
    from paper_2606_19557_gb300 import NEP, NepError
    spec = synth.SPECS["fcc32_t1"]
    nep = NEP(spec)
    b = synth.batch_fcc32(n_struct=2)
    with pytest.raises(NepError):
        nep.eval()  # no structures yet
    bad = synth.Batch(b.atom_off, b.pos.copy(), b.types, b.cell, 1)
    bad.pos[3, 1] = np.nan
    with pytest.raises(NepError):
        nep.set_structures_batch(bad)
    bt = synth.Batch(b.atom_off, b.pos, b.types + 1, b.cell, 1)
    with pytest.raises(NepError):
        nep.set_structures_batch(bt)
    bc = synth.Batch(b.atom_off, b.pos, b.types, np.zeros_like(b.cell), 1)
    with pytest.raises(NepError):
        nep.set_structures_batch(bc)
    bz = synth.Batch(np.array([0, 0, 64], np.int64), b.pos, b.types, b.cell, 1)
    with pytest.raises(NepError):
        nep.set_structures_batch(bz)
    nep.set_structures_batch(b)  # a valid batch still works afterwards
    with pytest.raises(NepError):
        nep.eval()  # no parameters yet
    P = oracle.num_params(spec)
    nep.set_params(torch.zeros(P), torch.ones(nep.n_des))
    E, F, W = nep.eval()
    assert np.all(np.isfinite(E.cpu().numpy()))


@pytest.mark.parametrize("name", ["fcc_bcc_t1", "alloy_t4"])
def test_plain_form_matches_oracle(name):
    """The per-structure baseline form computes the same loss and gradient."""
    from paper_2606_19557_gb300 import SCHED_PERSISTENT, SCHED_PLAIN
    c = get_case(name)
    c.nep.set_schedule(SCHED_PLAIN)
    try:
        l3, g = c.nep.loss_grad(c.E_ref, c.F_ref, c.W_ref)
        l3, g = l3.cpu().numpy(), g.cpu().numpy()
    finally:
        c.nep.set_schedule(SCHED_PERSISTENT)
    l3o, go = oracle.loss_grad(c.spec, c.theta, c.qs, c.batch, c.E_ref, c.F_ref, c.W_ref)[:2]
    np.testing.assert_allclose(l3, l3o, rtol=TOL)
    assert_grad_close(g, go, c.spec, TOL)


def test_shards_sum_to_full_batch():
    """Two shards evaluated with the whole batch's normalisers add up to the full pass."""
    from paper_2606_19557_gb300 import NEP, NepError, shard
    c = get_case("alloy_t4")
    b = c.batch
    hw = np.ones(b.n_struct, np.uint8)
    hw[1::4] = 0
    lam = (1.0, 2.0, 0.3)
    norms = shard.global_normalizers(b.counts(), hw)
    L = np.zeros(3)
    G = np.zeros(len(c.theta))
    for idx in shard.partition(b.counts(), 2):
        sub = b.subset(idx)
        a_idx = np.concatenate([np.arange(b.atom_off[i], b.atom_off[i + 1]) for i in idx])
        nep = NEP(c.spec)
        nep.set_structures_batch(sub)
        nep.set_params(torch.tensor(c.theta, dtype=torch.float32), torch.tensor(c.qs, dtype=torch.float32))
        nep.set_loss_normalizers(*norms)
        l3, g = nep.loss_grad(c.E_ref[idx], c.F_ref[a_idx], c.W_ref[idx], hw[idx], lam)
        L += l3.cpu().numpy()
        G += g.cpu().numpy().astype(np.float64)
        with pytest.raises(NepError):
            nep.set_loss_normalizers(-1.0, 0.0, 0.0)
        # back to the shard's own counts: now it is the shard's standalone loss
        nep.set_loss_normalizers()
        l3s, gs = nep.loss_grad(c.E_ref[idx], c.F_ref[a_idx], c.W_ref[idx], hw[idx], lam)
        l3o, go = oracle.loss_grad(c.spec, c.theta, c.qs, sub, c.E_ref[idx], c.F_ref[a_idx], c.W_ref[idx],
                                   hw[idx], lam)[:2]
        np.testing.assert_allclose(l3s.cpu().numpy(), l3o, rtol=TOL)
        assert_grad_close(gs.cpu().numpy(), go, c.spec, TOL)
        nep.close()
    l3o, go = oracle.loss_grad(c.spec, c.theta, c.qs, b, c.E_ref, c.F_ref, c.W_ref, hw, lam)[:2]
    np.testing.assert_allclose(L, l3o, rtol=TOL)
    assert rel(G, go) < TOL


def test_update_positions_matches_fresh_context():
    """New positions and cells for a cached batch (MD-style step): the rebuilt neighbour
    lists are the brute-force ones, E/F/W equal those of a fresh context bit for bit, and
    the loss gradient matches the oracle."""
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS["scale_t5"]
    b = synth.batch_scale(seed=17, n_struct=12, n_big=0)
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, 17)
    qs = f32(oracle.scale_from_range(oracle.descriptors(spec, theta, b)))
    nep = NEP(spec)
    nep.set_structures_batch(b)
    th_t, qs_t = torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32)
    nep.set_params(th_t, qs_t)
    nep.eval()
    rng = np.random.default_rng(3)
    strain = np.eye(3) + rng.uniform(-0.01, 0.01, size=(3, 3))
    pos2 = (np.asarray(b.pos, np.float64) @ strain.T + rng.normal(scale=0.05, size=b.pos.shape)).astype(np.float32)
    cell2 = (np.asarray(b.cell, np.float64).reshape(-1, 3, 3) @ strain.T).reshape(-1, 9).astype(np.float32)
    b2 = synth.Batch(b.atom_off, pos2.astype(np.float64), b.types, cell2.astype(np.float64), b.n_types)
    nep.update_positions(pos2, cell2)
    _check_neighbors(nep, b2, spec.rc_R, spec.rc_A)
    E, F, W = [x.cpu().numpy() for x in nep.eval()]
    fresh = NEP(spec)
    fresh.set_structures_batch(b2)
    fresh.set_params(th_t, qs_t)
    E2, F2, W2 = [x.cpu().numpy() for x in fresh.eval()]
    assert np.array_equal(E, E2) and np.array_equal(F, F2) and np.array_equal(W, W2)
    Eo, Fo, Wo = oracle.evaluate(spec, theta, qs, b2)
    assert rel(E, Eo) < TOL and rel(F, Fo) < TOL and rel(W, Wo) < TOL
    Er, Fr, Wr = synth.random_targets(b2, 5)
    l3, g = nep.loss_grad(Er, Fr, Wr)
    l3o, go = oracle.loss_grad(spec, theta, qs, b2, Er, Fr, Wr)[:2]
    np.testing.assert_allclose(l3.cpu().numpy(), l3o, rtol=TOL)
    assert_grad_close(g.cpu().numpy(), go, spec, TOL)



def test_update_positions_cells_kept_and_minibatches():
    """Positions-only updates (the cells' bin grids are kept and the schedules are built on
    the device), twice in a row, then an update with mini-batches set up (schedules built
    on the host): E/F/W, the loss and the gradient of the full batch and of a mini-batch
    equal those of a fresh context bit for bit."""
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS["scale_t5"]
    b = synth.batch_scale(seed=19, n_struct=16, n_big=0)
    P = oracle.num_params(spec)
    th = torch.tensor(synth.random_theta(P, 19), dtype=torch.float32)
    qs = torch.tensor(f32(oracle.scale_from_range(oracle.descriptors(spec, th.double().numpy(), b))),
                      dtype=torch.float32)
    Er, Fr, Wr = synth.random_targets(b, 20)
    lam = (1.0, 2.0, 0.3)
    nep = NEP(spec)
    nep.set_structures_batch(b)
    nep.set_params(th, qs)
    nep.eval()
    rng = np.random.default_rng(21)

    def fresh_for(pos, B=0):
        f = NEP(spec)
        f.set_structures_batch(synth.Batch(b.atom_off, pos.astype(np.float64), b.types, b.cell, b.n_types))
        f.set_params(th, qs)
        if B:
            f.minibatch_setup(B)
        return f

    def same(a, f):
        for x, y in zip(a.eval(), f.eval()):
            assert torch.equal(x, y)
        la, ga = a.loss_grad(Er, Fr, Wr, None, lam)
        lf, gf = f.loss_grad(Er, Fr, Wr, None, lam)
        assert torch.equal(la, lf) and torch.equal(ga, gf)

    for _ in range(2):
        pos = (np.asarray(b.pos) + rng.normal(scale=0.05, size=b.pos.shape)).astype(np.float32)
        nep.update_positions(pos)
        f = fresh_for(pos)
        same(nep, f)
        f.close()
    B = 5
    n = nep.minibatch_setup(B)
    pos = (np.asarray(b.pos) + rng.normal(scale=0.05, size=b.pos.shape)).astype(np.float32)
    nep.update_positions(pos)
    f = fresh_for(pos)
    same(nep, f)
    f.close()
    # the mini-batch launch shapes are chosen by timing: groups are checked against the oracle
    b2 = synth.Batch(b.atom_off, pos.astype(np.float64), b.types, b.cell, b.n_types)
    nep.set_targets(Er, Fr, Wr)
    theta = th.double().numpy()
    for m in range(n):
        s0, s1 = m * B, min(b.n_struct, (m + 1) * B)
        a0, a1 = b.atom_off[s0], b.atom_off[s1]
        la, ga = nep.minibatch_loss_grad(m, lam)
        lo, go = oracle.loss_grad(spec, theta, qs.double().numpy(), b2.subset(np.arange(s0, s1)), Er[s0:s1],
                                  Fr[a0:a1], Wr[s0:s1], None, lam)[:2]
        np.testing.assert_allclose(la.cpu().numpy(), lo, rtol=TOL)
        assert_grad_close(ga.cpu().numpy(), go, spec, TOL)
    nep.close()

def test_update_positions_candidate_lists():
    """Position updates with the cells kept go through candidate lists (every pair within
    r_c + skin of the positions of the last candidate scan): small moves are filtered from
    them, a move of more than half the skin rescans first.  After every update the lists
    equal the brute force's and those of a context that scans (skin 0) entry for entry, and
    E/F/W equal those of a fresh context bit for bit."""
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS["scale_t5"]
    b = synth.batch_scale(seed=23, n_struct=14, n_big=0)
    P = oracle.num_params(spec)
    th = torch.tensor(synth.random_theta(P, 23), dtype=torch.float32)
    qs = torch.tensor(f32(oracle.scale_from_range(oracle.descriptors(spec, th.double().numpy(), b))),
                      dtype=torch.float32)
    nep, scan = NEP(spec), NEP(spec)
    scan.set_skin(0.0)
    for x in (nep, scan):
        x.set_structures_batch(b)
        x.set_params(th, qs)
    rng = np.random.default_rng(29)
    pos = np.asarray(b.pos, np.float64)
    for step, sigma in enumerate((0.02, 0.03, 0.02, 0.4, 0.02)):  # the 0.4 A move rescans
        pos = pos + rng.normal(scale=sigma, size=pos.shape)
        p32 = pos.astype(np.float32)
        nep.update_positions(p32)
        scan.update_positions(p32)
        bs = synth.Batch(b.atom_off, p32.astype(np.float64), b.types, b.cell, b.n_types)
        _check_neighbors(nep, bs, spec.rc_R, spec.rc_A)
        for u, v in zip(nep.neighbors(), scan.neighbors()):
            assert torch.equal(u, v), step
        f = NEP(spec)
        f.set_structures_batch(bs)
        f.set_params(th, qs)
        for u, v in zip(nep.eval(), f.eval()):
            assert torch.equal(u, v), step
        f.close()
    nep.close()
    scan.close()


@pytest.mark.parametrize("name", ["nep44_t16", "nep88_t16"])
def test_table2_sixteen_species_models(name):
    """The paper's 16-element models (Table 2 sizes; 80 neurons, 4- and 5-body terms) on a
    16-species alloy batch: E/F/W, loss and gradient against the oracle."""
    from paper_2606_19557_gb300 import NEP
    spec = synth.SPECS[name]
    b = synth.batch_alloy(seed=61, n_struct=6, n_types=16, n_lo=24, n_hi=90)
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, 61)
    qs = f32(oracle.scale_from_range(oracle.descriptors(spec, theta, b)))
    nep = NEP(spec)
    nep.set_structures_batch(b)
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    E, F, W = [x.cpu().numpy() for x in nep.eval()]
    Eo, Fo, Wo = oracle.evaluate(spec, theta, qs, b)
    assert rel(E, Eo) < TOL and rel(F, Fo) < TOL and rel(W, Wo) < TOL
    Er, Fr, Wr = synth.random_targets(b, 62)
    lam = (1.0, 2.0, 0.3)
    l3, g = nep.loss_grad(Er, Fr, Wr, None, lam)
    l3o, go = oracle.loss_grad(spec, theta, qs, b, Er, Fr, Wr, None, lam)[:2]
    np.testing.assert_allclose(l3.cpu().numpy(), l3o, rtol=TOL)
    assert_grad_close(g.cpu().numpy(), go, spec, TOL)
    nep.autotune()  # every variant that fits the 16-species shared-memory tail
    g2 = nep.loss_grad(Er, Fr, Wr, None, lam)[1].cpu().numpy()
    assert_grad_close(g2, go, spec, TOL)



MODEL_VARIANTS = {
    # largest model the kernels take: n_max = basis = 11, l_max 4 with 4- and 5-body, 128 neurons
    "maximum": (synth.ModelSpec(3, 6.0, 4.5, 11, 11, 11, 11, 4, 1, 1, 128), 3),
    # smallest: one radial and one angular function of one basis term, l_max 0, one neuron
    "minimum": (synth.ModelSpec(2, 5.0, 4.0, 0, 0, 0, 0, 0, 0, 0, 1), 2),
    # l_max 1 with the 5-body term only
    "l1_5body": (synth.ModelSpec(2, 5.5, 4.0, 3, 2, 5, 4, 1, 0, 1, 16), 2),
    # l_max 2 with the 4-body term, angular cutoff equal to the radial one
    "l2_4body_equal_cutoffs": (synth.ModelSpec(2, 5.0, 5.0, 5, 3, 6, 5, 2, 1, 0, 20), 2),
}


@pytest.mark.parametrize("name", list(MODEL_VARIANTS))
def test_model_variants(name):
    """Corners of the model limits (n_max, basis_size, l_max, 4-/5-body flags, neurons,
    r_c^A = r_c^R) through E/F/W, the loss and the gradient."""
    from paper_2606_19557_gb300 import NEP
    spec, T = MODEL_VARIANTS[name]
    b = synth.batch_alloy(seed=81, n_struct=5, n_types=T, n_lo=20, n_hi=70)
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, 81)
    qs = f32(oracle.scale_from_range(oracle.descriptors(spec, theta, b)))
    nep = NEP(spec)
    nep.set_structures_batch(b)
    _check_neighbors(nep, b, spec.rc_R, spec.rc_A)
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    E, F, W = [x.cpu().numpy() for x in nep.eval()]
    Eo, Fo, Wo = oracle.evaluate(spec, theta, qs, b)
    assert rel(E, Eo) < TOL and rel(F, Fo) < TOL and rel(W, Wo) < TOL
    Er, Fr, Wr = synth.random_targets(b, 82)
    l3, g = nep.loss_grad(Er, Fr, Wr, None, (1.0, 1.0, 0.1))
    l3o, go = oracle.loss_grad(spec, theta, qs, b, Er, Fr, Wr, None, (1.0, 1.0, 0.1))[:2]
    np.testing.assert_allclose(l3.cpu().numpy(), l3o, rtol=TOL)
    assert_grad_close(g.cpu().numpy(), go, spec, TOL)
    nep.close()


class _SpecZBL:
    """A model spec with the ZBL short-range term (switch radii, atomic numbers)."""

    def __init__(self, base, zbl):
        for k in ("n_types", "rc_R", "rc_A", "n_max_R", "n_max_A", "basis_R", "basis_A", "l_max", "has_4b",
                  "has_5b", "n_neu"):
            setattr(self, k, getattr(base, k))
        self.zbl = zbl


@pytest.mark.parametrize("name,zbl", [("alloy_t4", (1.5, 2.4, [29.0, 28.0, 26.0, 13.0])),
                                      ("scale_t5", (0.0, 2.2, [6.0, 14.0, 8.0, 1.0, 79.0]))])
def test_zbl_matches_oracle(name, zbl):
    """E, F, W, loss and gradient with the ZBL term on (Sec. "Training"), on liquid-like
    structures whose closest pairs fall inside the switch and below r1."""
    from paper_2606_19557_gb300 import NEP
    spec = _SpecZBL(synth.SPECS[name], zbl)
    b = synth.batch_alloy(seed=91, n_struct=8, n_types=spec.n_types, n_lo=12, n_hi=60)
    P = oracle.num_params(spec)
    theta = synth.random_theta(P, 91)
    qs = f32(oracle.scale_from_range(oracle.descriptors(spec, theta, b)))
    i, j, S, ang = oracle.neighbors(b, spec.rc_R, spec.rc_A)
    d = b.pos[j] - b.pos[i] + np.einsum("pk,pkx->px", S.astype(np.float64),
                                        b.cell.reshape(-1, 3, 3)[np.searchsorted(b.atom_off, i, side="right") - 1])
    r = np.linalg.norm(d, axis=1)
    assert np.sum(r < zbl[1]) > 20  # the term is exercised
    nep = NEP(spec)
    nep.set_structures_batch(b)
    nep.set_params(torch.tensor(theta, dtype=torch.float32), torch.tensor(qs, dtype=torch.float32))
    E, F, W = [x.cpu().numpy() for x in nep.eval()]
    Eo, Fo, Wo = oracle.evaluate(spec, theta, qs, b)
    assert rel(E, Eo) < TOL and rel(F, Fo) < TOL and rel(W, Wo) < TOL
    E0 = oracle.evaluate(_SpecZBL(synth.SPECS[name], None), theta, qs, b)[0]
    assert rel(E0, Eo) > 1e-3  # the ZBL term changes the energies well beyond the tolerance
    Er, Fr, Wr = synth.random_targets(b, 92)
    lam = (1.0, 1.0, 0.1)
    l3, g = nep.loss_grad(Er, Fr, Wr, None, lam)
    l3o, go = oracle.loss_grad(spec, theta, qs, b, Er, Fr, Wr, None, lam)[:2]
    np.testing.assert_allclose(l3.cpu().numpy(), l3o, rtol=TOL)
    assert_grad_close(g.cpu().numpy(), go, spec, TOL)
    # switched off again: the plain model
    nep.set_zbl(0.0, 0.0)
    E2 = nep.eval()[0].cpu().numpy()
    assert rel(E2, E0) < TOL
    nep.close()
