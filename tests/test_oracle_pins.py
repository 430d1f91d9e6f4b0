"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

CPU only.  Each test checks one place where a plausible mistake (dropped term,
wrong sign or index, transposed operand, wrong normalisation) would show:
  * Table 2 parameter counts (printed in the paper);
  * coordination-shell counts of perfect lattices (textbook);
  * Chebyshev basis against the trigonometric form, and the stated property that
    f_k and f_k' vanish at r_c (Methods);
  * orthonormality of the real harmonics by quadrature, the addition theorem, and
    agreement with scipy's complex harmonics;
  * the 4-body invariant against Wigner 3j symbols (sympy) contracted with complex
    moments (scipy);
  * a dimer's closed form;
  * central finite differences for F, W and dL/dtheta;
  * translation / rotation / permutation invariance (Methods, last paragraph of
    "NEP descriptors"), zero net force, symmetric virial;
  * teacher = student gives L = 0 and a zero gradient; q linear in c^R.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2606_19557_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


class Spec:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def spec(n_types=1, rc_R=5.0, rc_A=4.0, n_max_R=4, n_max_A=4, basis_R=8, basis_A=8, l_max=4, has_4b=0, has_5b=0,
         n_neu=10):
    return Spec(n_types=n_types, rc_R=rc_R, rc_A=rc_A, n_max_R=n_max_R, n_max_A=n_max_A, basis_R=basis_R,
                basis_A=basis_A, l_max=l_max, has_4b=has_4b, has_5b=has_5b, n_neu=n_neu)


def one_batch(pos, cell, types=None):
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    n = pos.shape[0]
    return synth.Batch(np.array([0, n], np.int64), pos, np.zeros(n, np.int32) if types is None else
                       np.asarray(types, np.int32), np.asarray(cell, np.float64).reshape(1, 9), 1)


def fd_batch(batch):
    """Copy with float64 positions/cells (finite differences perturb them in FP64)."""
    return synth.Batch(batch.atom_off.copy(), batch.pos.astype(np.float64), batch.types.copy(),
                       batch.cell.astype(np.float64), batch.n_types)


# ------------------------------------------------------------------ parameter counts

def test_table2_parameter_counts():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table2_param_counts.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        T, nR, nA, bR, bA, L, h4, h5, nn, P = map(int, r[1:])
        s = spec(n_types=T, n_max_R=nR, n_max_A=nA, basis_R=bR, basis_A=bA, l_max=L, has_4b=h4, has_5b=h5, n_neu=nn)
        assert oracle.num_params(s) == P, r[0]


def test_config_parameter_counts():
    expect = {"fcc32_t1": 361, "fcc_bcc_t1": 1051, "alloy_t4": 5281, "scale_t5": 16601, "carbon_table1": 6903}
    for k, P in expect.items():
        assert oracle.num_params(synth.SPECS[k]) == P, k


# ------------------------------------------------------------------ neighbour lists

def _lattice_batch(kind, a, reps, primitive=False):
    if primitive:
        cell = 0.5 * a * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]], float)
        return one_batch([[0.1, 0.2, 0.3]], cell)
    frac, cell = synth._lattice(kind, reps, a)
    return one_batch(frac @ cell, cell)


@pytest.mark.parametrize("reps", [(1, 1, 1), (2, 2, 2), (3, 2, 2)])
def test_shell_counts(reps):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "coordination_shells.txt")) if l.strip() and l[0] != "#"]
    for kind, a, rc, cnt in rows:
        b = _lattice_batch(kind, float(a), reps)
        i, j, S, ang = oracle.neighbors(b, float(rc), float(rc))
        per_atom = np.bincount(i, minlength=b.n_atoms)
        assert np.all(per_atom == int(cnt)), (kind, a, rc, reps, per_atom[:4])


def test_primitive_triclinic_cell_self_images():
    # one-atom FCC primitive cell: every neighbour is an image of the atom itself
    b = _lattice_batch("fcc", 3.6, None, primitive=True)
    i, j, S, ang = oracle.neighbors(b, 6.0, 4.0)
    assert len(i) == 78 and np.all(j == 0) and int(ang.sum()) == 18
    assert len({tuple(s) for s in S}) == 78


def test_neighbor_list_symmetric_and_unique():
    b = synth.batch_alloy(seed=11, n_struct=6, n_types=3, n_lo=2, n_hi=40)
    i, j, S, ang = oracle.neighbors(b, 6.0, 4.0)
    keys = set(zip(i.tolist(), j.tolist(), map(tuple, S.tolist())))
    assert len(keys) == len(i)
    for a, bb, s in list(keys)[:2000]:
        assert (bb, a, tuple(-x for x in s)) in keys


# ------------------------------------------------------------------ basis functions

def test_chebyshev_basis_trig_form_and_cutoff():
    rc, K = 5.0, 12
    for r in np.linspace(0.3, 4.99, 37):
        f, fp = oracle.basis(r, rc, K)
        x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
        fc = 0.5 * (math.cos(math.pi * r / rc) + 1.0)
        expect = 0.5 * (np.cos(np.arange(K) * math.acos(x)) + 1.0) * fc
        np.testing.assert_allclose(f, expect, rtol=1e-12, atol=1e-14)
        h = 1e-6
        fpn = (oracle.basis(r + h, rc, K)[0] - oracle.basis(r - h, rc, K)[0]) / (2 * h)
        np.testing.assert_allclose(fp, fpn, rtol=1e-6, atol=1e-8)
    f, fp = oracle.basis(rc, rc, K)
    assert np.all(np.abs(f) < 1e-15) and np.all(np.abs(fp) < 1e-12)
    f, fp = oracle.basis(rc + 0.1, rc, K)
    assert np.all(f == 0) and np.all(fp == 0)
    f, _ = oracle.basis(0.0, rc, K)  # x = 1: T_k = 1 and f_c = 1
    np.testing.assert_allclose(f, np.ones(K), rtol=1e-14)


# ------------------------------------------------------------------ harmonics

def _sphere_quadrature(n=24):
    xg, wg = np.polynomial.legendre.leggauss(n)
    phi = 2 * np.pi * np.arange(2 * n) / (2 * n)
    z, p = np.meshgrid(xg, phi, indexing="ij")
    w = np.repeat(wg[:, None], 2 * n, 1) * (2 * np.pi / (2 * n))
    s = np.sqrt(1 - z ** 2)
    return np.stack([s * np.cos(p), s * np.sin(p), z], -1).reshape(-1, 3), w.reshape(-1)


def test_real_harmonics_orthonormal():
    u, w = _sphere_quadrature()
    Y = np.stack([oracle.ylm(x)[0] for x in u])
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(24), atol=1e-12)


def test_real_harmonics_addition_theorem_and_scipy():
    from scipy.special import eval_legendre, sph_harm_y
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = rng.normal(size=3), rng.normal(size=3) * 3.0
        Ya, Yb = oracle.ylm(a)[0], oracle.ylm(b)[0]
        ua, ub = a / np.linalg.norm(a), b / np.linalg.norm(b)
        for l in range(1, 5):
            sl = slice(l * l - 1, l * l - 1 + 2 * l + 1)
            lhs = Ya[sl] @ Yb[sl]
            assert abs(lhs - (2 * l + 1) / (4 * np.pi) * eval_legendre(l, ua @ ub)) < 1e-13
            # |real Y_l.|^2 summed equals |complex Y_l.|^2 summed, pointwise per |m|
            th, ph = math.acos(ua[2]), math.atan2(ua[1], ua[0])
            for m in range(0, l + 1):
                c = sph_harm_y(l, m, th, ph)
                real_pair = Ya[l * l - 1 + l + m] ** 2 + (Ya[l * l - 1 + l - m] ** 2 if m > 0 else 0.0)
                assert abs(real_pair - (2 if m > 0 else 1) * abs(c) ** 2) < 1e-12


def test_real_harmonics_gradient_fd():
    rng = np.random.default_rng(1)
    for _ in range(10):
        d = rng.normal(size=3) * 2.5
        _, g = oracle.ylm(d)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            num = (oracle.ylm(d + e)[0] - oracle.ylm(d - e)[0]) / (2 * h)
            np.testing.assert_allclose(g[:, a], num, atol=1e-8)


# ------------------------------------------------------------------ invariants of one atom

def _centre_environment(rng, n_nb, rmin=1.5, rmax=3.8):
    u = rng.normal(size=(n_nb, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = rng.uniform(rmin, rmax, size=n_nb)
    pos = np.vstack([[15.0, 15.0, 15.0], 15.0 + u * r[:, None]])
    return pos, np.eye(3) * 30.0


def _g_weights(s, theta, r_list, which="A", ti=0, tj=0):
    P = oracle.num_params(s)
    NR, KR, NA, KA = s.n_max_R + 1, s.basis_R + 1, s.n_max_A + 1, s.basis_A + 1
    ND = NR + NA * (s.l_max + s.has_4b + s.has_5b)
    T, NN = s.n_types, s.n_neu
    o_cR = T * NN * ND + 2 * T * NN + 1
    o_cA = o_cR + T * T * NR * KR
    assert o_cA + T * T * NA * KA == P
    if which == "A":
        c = theta[o_cA:].reshape(T, T, NA, KA)[ti, tj]
        rc, K = s.rc_A, KA
    else:
        c = theta[o_cR:o_cA].reshape(T, T, NR, KR)[ti, tj]
        rc, K = s.rc_R, KR
    return np.array([c @ oracle.basis(r, rc, K)[0] for r in r_list])  # [n_nb, N]


def test_q3_addition_theorem_and_q5():
    from scipy.special import eval_legendre
    s = spec(l_max=4, has_4b=1, has_5b=1)
    rng = np.random.default_rng(2)
    theta = synth.random_theta(oracle.num_params(s), 3)
    pos, cell = _centre_environment(rng, 9)
    q = oracle.descriptors(s, theta, one_batch(pos, cell))[0]
    d = pos[1:] - pos[0]
    r = np.linalg.norm(d, axis=1)
    u = d / r[:, None]
    g = _g_weights(s, theta, r)
    NR, NA = 5, 5
    for l in range(1, 5):
        Pl = eval_legendre(l, u @ u.T)
        for n in range(NA):
            expect = (2 * l + 1) / (4 * np.pi) * g[:, n] @ Pl @ g[:, n]
            assert abs(q[NR + (l - 1) * NA + n] - expect) < 1e-12 * max(1.0, abs(expect))
    for n in range(NA):
        assert abs(q[NR + 5 * NA + n] - q[NR + n] ** 2) < 1e-12 * max(1.0, q[NR + n] ** 2)
    # radial descriptor: plain sum of g_n over neighbours
    gR = _g_weights(s, theta, r, which="R")
    np.testing.assert_allclose(q[:NR], gR.sum(0), rtol=1e-12, atol=1e-13)


def test_q4_matches_wigner_3j_contraction():
    sympy = pytest.importorskip("sympy")
    from sympy.physics.wigner import wigner_3j
    from scipy.special import sph_harm_y
    tj = {}
    for m1 in range(-2, 3):
        for m2 in range(-2, 3):
            m3 = -m1 - m2
            if abs(m3) <= 2:
                tj[(m1, m2, m3)] = float(wigner_3j(2, 2, 2, m1, m2, m3))
    s = spec(l_max=2, has_4b=1)
    rng = np.random.default_rng(4)
    theta = synth.random_theta(oracle.num_params(s), 5)
    NR, NA = 5, 5
    for trial in range(5):
        pos, cell = _centre_environment(rng, 4 + trial)
        q = oracle.descriptors(s, theta, one_batch(pos, cell))[0]
        d = pos[1:] - pos[0]
        r = np.linalg.norm(d, axis=1)
        u = d / r[:, None]
        g = _g_weights(s, theta, r)
        th, ph = np.arccos(u[:, 2]), np.arctan2(u[:, 1], u[:, 0])
        for n in range(NA):
            A = {m: np.sum(g[:, n] * sph_harm_y(2, m, th, ph)) for m in range(-2, 3)}
            val = sum(c * A[m1] * A[m2] * A[m3] for (m1, m2, m3), c in tj.items())
            assert abs(val.imag) < 1e-12
            got = q[NR + 2 * NA + n]
            assert abs(got - val.real) < 1e-11 * max(1.0, abs(val.real)), (n, got, val)


def test_dimer_closed_form():
    s = spec(rc_R=6.0, rc_A=4.0, has_4b=1, has_5b=1, n_neu=7)
    theta = synth.random_theta(oracle.num_params(s), 8)
    for r in (1.9, 2.7, 3.5, 4.5):
        pos = np.array([[6.0, 6.0, 6.0], [6.0 + r * 0.6, 6.0 + r * 0.8, 6.0]])
        b = one_batch(pos, np.eye(3) * 12.0)
        q = oracle.descriptors(s, theta, b)[0]
        gR = _g_weights(s, theta, [r], which="R")[0]
        np.testing.assert_allclose(q[:5], gR, rtol=1e-12, atol=1e-14)
        gA = _g_weights(s, theta, [r])[0] if r < 4.0 else np.zeros(5)
        for l in range(1, 5):
            np.testing.assert_allclose(q[5 + (l - 1) * 5:5 + l * 5], (2 * l + 1) / (4 * np.pi) * gA ** 2,
                                       rtol=1e-12, atol=1e-14)
        # one bond along u: M = g (u u^T - I/3) has tr(M^3) = 2 g^3 / 9
        np.testing.assert_allclose(q[25:30], oracle.kappa4() * 2.0 / 9.0 * gA ** 3, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(q[30:35], (3 / (4 * np.pi) * gA ** 2) ** 2, rtol=1e-12, atol=1e-14)


def test_kappa_value():
    # (2 2 2; 0 0 0) Y20(z)^3 = KAPPA tr(Q(z)^3) with Q(z) = diag(-1/3, -1/3, 2/3)
    y20 = math.sqrt(5 / (4 * math.pi))
    assert abs(-math.sqrt(2 / 35) * y20 ** 3 - oracle.kappa4() * 2.0 / 9.0) < 1e-15


# ------------------------------------------------------------------ derivatives

def _small_case(name, seed=21, n_struct=3, n_lo=6, n_hi=14):
    s = synth.SPECS[name]
    if name == "fcc32_t1":
        b = synth.batch_fcc32(n_struct=1)
    else:
        b = synth.batch_alloy(seed=seed, n_struct=n_struct, n_types=s.n_types, n_lo=n_lo, n_hi=n_hi)
    b = fd_batch(b)
    theta = synth.random_theta(oracle.num_params(s), seed)
    qs = oracle.scale_from_range(oracle.descriptors(s, theta, b))
    return s, b, theta, qs


@pytest.mark.parametrize("name", ["fcc32_t1", "alloy_t4", "scale_t5"])
def test_forces_finite_difference(name):
    s, b, theta, qs = _small_case(name)
    E, F, W = oracle.evaluate(s, theta, qs, b)
    off = b.atom_off
    h = 1e-5
    rng = np.random.default_rng(0)
    for i in rng.choice(b.n_atoms, size=min(6, b.n_atoms), replace=False):
        st = int(np.searchsorted(off, i, side="right") - 1)
        for a in range(3):
            bp, bm = fd_batch(b), fd_batch(b)
            bp.pos[i, a] += h
            bm.pos[i, a] -= h
            Ep = oracle.evaluate(s, theta, qs, bp)[0][st]
            Em = oracle.evaluate(s, theta, qs, bm)[0][st]
            assert abs(-(Ep - Em) / (2 * h) - F[i, a]) < 2e-7 * max(1.0, np.abs(F).max())


@pytest.mark.parametrize("name", ["fcc32_t1", "alloy_t4", "scale_t5"])
def test_virial_finite_difference(name):
    s, b, theta, qs = _small_case(name)
    E, F, W = oracle.evaluate(s, theta, qs, b)
    h = 1e-6
    for st in range(b.n_struct):
        a0, a1 = b.atom_off[st], b.atom_off[st + 1]
        for ab in range(9):
            eps = np.zeros(9)
            eps[ab] = h
            out = []
            for sgn in (1, -1):
                Fm = np.eye(3) + sgn * eps.reshape(3, 3)
                bb = fd_batch(b)
                bb.pos[a0:a1] = bb.pos[a0:a1] @ Fm.T
                bb.cell[st] = (bb.cell[st].reshape(3, 3) @ Fm.T).reshape(9)
                out.append(oracle.evaluate(s, theta, qs, bb)[0][st])
            assert abs(-(out[0] - out[1]) / (2 * h) - W[st, ab]) < 1e-6 * max(1.0, np.abs(W).max())


@pytest.mark.parametrize("name", ["fcc32_t1", "alloy_t4", "scale_t5"])
def test_loss_gradient_finite_difference(name):
    s, b, theta, qs = _small_case(name, n_struct=2, n_lo=8, n_hi=12)
    Er, Fr, Wr = synth.random_targets(b, 9)
    has_W = np.array([1, 0] * (b.n_struct // 2) + [1] * (b.n_struct % 2), np.uint8)
    lam = (1.0, 2.0, 0.3)
    loss3, g = oracle.loss_grad(s, theta, qs, b, Er, Fr, Wr, has_W, lam)[:2]
    P = len(theta)
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([rng.choice(P, size=min(P, 60), replace=False), [P - 1, 0]]))
    # make sure every block (w0, b0, w1, b1, cR, cA) is hit
    NR, KR, NA, KA = s.n_max_R + 1, s.basis_R + 1, s.n_max_A + 1, s.basis_A + 1
    ND = NR + NA * (s.l_max + s.has_4b + s.has_5b)
    T, NN = s.n_types, s.n_neu
    o_b1 = T * NN * ND + 2 * T * NN
    idx = np.unique(np.concatenate([idx, [T * NN * ND, T * NN * ND + T * NN, o_b1, o_b1 + 1, o_b1 + 1 + T * T * NR * KR]]))
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        Lp = oracle.loss_value(oracle.loss_grad(s, tp, qs, b, Er, Fr, Wr, has_W, lam)[0], lam)
        Lm = oracle.loss_value(oracle.loss_grad(s, tm, qs, b, Er, Fr, Wr, has_W, lam)[0], lam)
        assert abs((Lp - Lm) / (2 * h) - g[k]) < 1e-6 * max(1.0, np.abs(g).max()), k


def test_double_backward_reference_agrees():
    from oracle import torch_ref
    for name in ("fcc32_t1", "alloy_t4", "scale_t5"):
        s, b, theta, qs = _small_case(name, n_struct=3, n_lo=10, n_hi=20)
        pairs = oracle.neighbors(b, s.rc_R, s.rc_A)
        Er, Fr, Wr = synth.random_targets(b, 4)
        has_W = np.ones(b.n_struct, np.uint8)
        has_W[0] = 0
        l3, g = oracle.loss_grad(s, theta, qs, b, Er, Fr, Wr, has_W)[:2]
        l3t, gt = torch_ref.loss_grad(s, b, pairs, theta, qs, Er, Fr, Wr, has_W)
        np.testing.assert_allclose(l3, l3t, rtol=1e-12)
        assert np.linalg.norm(g - gt) <= 1e-11 * np.linalg.norm(g)


# ------------------------------------------------------------------ invariances

def _rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


@pytest.mark.parametrize("name", ["alloy_t4", "scale_t5"])
def test_invariances_and_conservation(name):
    s, b, theta, qs = _small_case(name, n_struct=3, n_lo=10, n_hi=30)
    E, F, W = oracle.evaluate(s, theta, qs, b)
    # zero net force per structure, symmetric virial
    for st in range(b.n_struct):
        a0, a1 = b.atom_off[st], b.atom_off[st + 1]
        assert np.abs(F[a0:a1].sum(0)).max() < 1e-11 * max(1.0, np.abs(F).max())
        Wm = W[st].reshape(3, 3)
        assert np.abs(Wm - Wm.T).max() < 1e-11 * max(1.0, np.abs(W).max())
    rng = np.random.default_rng(3)
    # translation
    bt = fd_batch(b)
    bt.pos += rng.normal(size=3) * 3.7
    Et, Ft, Wt = oracle.evaluate(s, theta, qs, bt)
    np.testing.assert_allclose(Et, E, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(Ft, F, rtol=1e-9, atol=1e-10)
    # rotation of positions and cell: E invariant, F -> R F, W -> R W R^T
    R = _rotation(rng)
    br = fd_batch(b)
    br.pos = br.pos @ R.T
    br.cell = (br.cell.reshape(-1, 3, 3) @ R.T).reshape(-1, 9)
    Er, Frr, Wr = oracle.evaluate(s, theta, qs, br)
    np.testing.assert_allclose(Er, E, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(Frr, F @ R.T, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(Wr.reshape(-1, 3, 3), R @ W.reshape(-1, 3, 3) @ R.T, rtol=1e-9, atol=1e-9)
    # permutation of atoms inside each structure (species travel with the atoms)
    perm = np.concatenate([b.atom_off[st] + rng.permutation(b.atom_off[st + 1] - b.atom_off[st])
                           for st in range(b.n_struct)])
    bp = fd_batch(b)
    bp.pos = bp.pos[perm]
    bp.types = bp.types[perm]
    Ep, Fp, Wp = oracle.evaluate(s, theta, qs, bp)
    np.testing.assert_allclose(Ep, E, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(Fp, F[perm], rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(Wp, W, rtol=1e-9, atol=1e-9)


def test_teacher_gives_zero_loss_and_gradient():
    s, b, theta, qs = _small_case("alloy_t4", n_struct=2, n_lo=10, n_hi=16)
    E, F, W = oracle.evaluate(s, theta, qs, b)
    loss3, g = oracle.loss_grad(s, theta, qs, b, E, F, W)[:2]
    assert np.all(loss3 == 0.0)
    assert np.all(g == 0.0)


def test_radial_descriptor_linear_in_c():
    s, b, theta, qs = _small_case("alloy_t4", n_struct=2, n_lo=10, n_hi=16)
    NR = s.n_max_R + 1
    q = oracle.descriptors(s, theta, b)
    NA, KA = s.n_max_A + 1, s.basis_A + 1
    T = s.n_types
    nA = T * T * NA * KA
    th2 = theta.copy()
    th2[-nA - T * T * NR * (s.basis_R + 1):-nA] *= -2.5
    q2 = oracle.descriptors(s, th2, b)
    np.testing.assert_allclose(q2[:, :NR], -2.5 * q[:, :NR], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(q2[:, NR:], q[:, NR:], rtol=0, atol=0)


# ------------------------------------------------------------------ hand-worked fixtures

def _fixture(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            rows.setdefault(k, []).append(v)
    return rows


def _frac(x):
    from fractions import Fraction
    return float(Fraction(x))


def loss_fixture():
    """Inputs and hand-worked Eq. "loss" values of tests/golden/loss_terms_b1_only.txt: three
    structures (a dimer, a triangle, one atom) in 12 A cells and a model whose only nonzero
    parameter is b1."""
    f = _fixture("loss_terms_b1_only.txt")
    nat = [int(x) for x in f["natoms"][0]]
    geo = {1: [[6.0, 6.0, 6.0]], 2: [[5.0, 6.0, 6.0], [7.1, 6.0, 6.0]],
           3: [[5.0, 5.0, 6.0], [7.0, 5.2, 6.0], [6.1, 6.9, 6.3]]}
    pos = np.concatenate([np.array(geo[n], np.float64) for n in nat])
    off = np.concatenate([[0], np.cumsum(nat)]).astype(np.int64)
    cell = np.tile((np.eye(3) * 12.0).reshape(9), (len(nat), 1))
    batch = synth.Batch(off, pos, np.zeros(pos.shape[0], np.int32), cell, 1)
    s = synth.SPECS["fcc_bcc_t1"]
    P = oracle.num_params(s)
    ND = oracle.num_descriptors(s)
    i_b1 = s.n_types * (ND + 2) * s.n_neu
    theta = np.zeros(P)
    theta[i_b1] = float(f["b1"][0][0])
    return {"spec": s, "batch": batch, "theta": theta, "i_b1": i_b1, "qs": np.ones(ND),
            "E_ref": np.array([float(x) for x in f["E_ref"][0]]),
            "F_ref": np.array([[float(x) for x in r] for r in f["F_ref"]]),
            "W_ref": np.array([[float(x) for x in r] for r in f["W_ref"]]),
            "has_W": np.array([int(x) for x in f["has_W"][0]], np.uint8),
            "lam": tuple(float(x) for x in f["lam"][0]),
            "loss3": np.array([_frac(x) for x in f["loss3"][0]]), "dL_db1": _frac(f["dL_db1"][0][0])}


def test_loss_terms_hand_worked():
    """Eq. "loss" normalisers (per-atom energy and virial residuals, 1/(3 N_a), N_s^V of the
    structures with virials) and the sign of b1, against the hand-worked fixture."""
    fx = loss_fixture()
    loss3, g, E, F, W = oracle.loss_grad(fx["spec"], fx["theta"], fx["qs"], fx["batch"], fx["E_ref"], fx["F_ref"],
                                         fx["W_ref"], fx["has_W"], fx["lam"])
    np.testing.assert_allclose(E, -0.5 * fx["batch"].counts(), rtol=0, atol=1e-15)
    assert np.all(F == 0.0) and np.all(W == 0.0)
    np.testing.assert_allclose(loss3, fx["loss3"], rtol=1e-14)
    assert abs(g[fx["i_b1"]] - fx["dL_db1"]) < 1e-14
    rest = np.delete(g, fx["i_b1"])
    assert np.all(rest == 0.0)


def dimer_fixture():
    f = _fixture("dimer_one_neuron.txt")
    s = spec(rc_R=float(f["rc_R"][0][0]), rc_A=float(f["rc_A"][0][0]), n_max_R=0, n_max_A=0, basis_R=0, basis_A=0,
             l_max=0, n_neu=1)
    pos = np.array([[float(x) for x in f["pos1"][0]], [float(x) for x in f["pos2"][0]]])
    return {"spec": s, "batch": one_batch(pos, np.eye(3) * 12.0),
            "theta": np.array([float(x) for x in f["theta"][0]]),
            "qs": np.array([float(x) for x in f["q_scale"][0]])}


def dimer_closed_form():
    """E_s, F_2 (x component) and W_xx of the one-neuron dimer (closed forms of the fixture)."""
    t = math.tanh(0.25)
    sech2 = 1.0 - t * t
    return 4.0 * t - 0.2, 0.5 * math.pi * sech2, math.pi * sech2


def test_network_signs_one_neuron_dimer():
    """Signs of Eq. "ann" (z = w0 q~ - b0, E_i = w1 tanh z - b1), F = -dE/dr and the virial
    convention, against closed forms of a one-neuron model on a dimer."""
    fx = dimer_fixture()
    assert oracle.num_params(fx["spec"]) == 6
    E, F, W = oracle.evaluate(fx["spec"], fx["theta"], fx["qs"], fx["batch"])
    Es, F2, Wxx = dimer_closed_form()
    assert abs(E[0] - Es) < 1e-14
    np.testing.assert_allclose(F, [[-F2, 0, 0], [F2, 0, 0]], rtol=0, atol=1e-14)
    np.testing.assert_allclose(W[0], [Wxx, 0, 0, 0, 0, 0, 0, 0, 0], rtol=0, atol=1e-14)


def _wide_brute_force(pos, cell, rc):
    """Every (i, j, S) with S in [-K, K]^3 for a K well beyond the needed range, kept by the
    float predicate of the neighbour build: d = r_j + S h - r_i in FP64 rounded to float,
    (dx dx + dy dy) + dz dz < rc rc in float without fused operations."""
    inv = np.linalg.inv(cell)
    w = 1.0 / np.linalg.norm(inv, axis=0)
    K = int(math.ceil(rc / w.min())) + 3
    rng = np.arange(-K, K + 1)
    S = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    shift = S.astype(np.float64) @ cell
    rc32 = np.float32(rc)
    out = set()
    for i in range(pos.shape[0]):
        for j in range(pos.shape[0]):
            d = (pos[j] - pos[i])[None, :] + shift
            d32 = d.astype(np.float32)
            r2 = (d32[:, 0] * d32[:, 0] + d32[:, 1] * d32[:, 1]) + d32[:, 2] * d32[:, 2]
            keep = r2 < rc32 * rc32
            for s in S[keep]:
                if i != j or s.any():
                    out.add((i, j, tuple(int(x) for x in s)))
    return out


def test_image_range_covers_float_predicate():
    """The brute-force enumeration takes |S_a| <= ceil(rc/w_a + span_a).  A pair outside that
    range has |d| >= w_a (ceil(rc/w_a + span_a) + 1 - span_a) >= rc + w_a, far beyond the
    float predicate's slack (kept pairs have |d| < rc (1 + 3 2^-24)).  Checked against an
    enumeration three shells wider on narrow triclinic cells whose atoms span the cell,
    including pairs placed within a few ulp of the cutoff."""
    rng = np.random.default_rng(7)
    for case in range(6):
        w = rng.uniform(1.3, 3.0)
        cell = np.diag([w, rng.uniform(1.3, 4.0), rng.uniform(2.0, 5.0)])
        cell = cell @ (np.eye(3) + 0.15 * rng.uniform(-1, 1, (3, 3)))
        n = 3
        frac = rng.uniform(0.0, 1.0, (n, 3))
        frac[0, 0], frac[1, 0] = 0.0, 0.999
        pos = frac @ cell
        rc = 4.0
        if case % 2:  # put one image pair at the cutoff: the displacement scaled to |d| = rc
            d = pos[1] + cell[0] * 2 - pos[0]
            pos[1] = pos[0] + d * (rc / np.linalg.norm(d)) - cell[0] * 2
        pos = pos.astype(np.float32).astype(np.float64)
        b = one_batch(pos, cell)
        i, j, S, _ = oracle.neighbors(b, rc, 3.0)
        got = set(zip(i.tolist(), j.tolist(), map(tuple, S.tolist())))
        assert got == _wide_brute_force(pos, cell, rc), case


# ------------------------------------------------------------------ ZBL short-range term

E2_4PI_EPS0 = 14.399645  # e^2 / (4 pi eps_0) in eV A (CODATA)


def zbl_spec(Z, r1=1.0, r2=2.0, n_types=2):
    s = spec(n_types=n_types, rc_R=5.0, rc_A=4.0, n_max_R=3, n_max_A=3, basis_R=5, basis_A=5, l_max=4, has_4b=1,
             has_5b=1, n_neu=6)
    s.zbl = (r1, r2, list(Z))
    return s


def _dimer_energy(s, r, types, theta=None):
    pos = np.array([[6.0, 6.0, 6.0], [6.0 + r, 6.0, 6.0]])
    b = one_batch(pos, np.eye(3) * 12.0, types)
    th = np.zeros(oracle.num_params(s)) if theta is None else theta
    return oracle.evaluate(s, th, np.ones(oracle.num_descriptors(s)), b)


def test_zbl_coulomb_limit():
    """At short range the screened repulsion of a pair tends to the bare Coulomb energy
    Z_i Z_j e^2 / (4 pi eps_0 r): the universal screening function is 1 at the origin (its
    four published coefficients add up to 1.00007).  Only the ZBL term is nonzero here
    (all network parameters zero)."""
    Z = (14.0, 6.0)
    s = zbl_spec(Z)
    g = []
    for r in (1e-4, 2e-4):
        E = _dimer_energy(s, r, [0, 1])[0][0]
        g.append(E * r / (E2_4PI_EPS0 * Z[0] * Z[1]))
    g0 = 2 * g[0] - g[1]  # linear extrapolation to r = 0
    assert abs(g0 - 1.0) < 1e-4
    assert g[0] < g0  # screening lowers the energy below the bare Coulomb value


def test_zbl_universal_scaling_and_switch():
    """The screened energy depends on the pair only through Z_i Z_j / r and the universal
    length r (Z_i^0.23 + Z_j^0.23): two species pairs at the same reduced distance give the
    same phi.  Inside r1 the switch is 1; at and beyond r2 the term is exactly zero, and it
    goes to zero smoothly (energy and force continuous)."""
    Za, Zb = (29.0, 29.0), (8.0, 1.0)
    sa, sb = zbl_spec(Za, r1=3.0, r2=4.0), zbl_spec(Zb, r1=3.0, r2=4.0)
    ua = Za[0] ** 0.23 + Za[1] ** 0.23
    ub = Zb[0] ** 0.23 + Zb[1] ** 0.23
    for x in (0.3, 1.0, 2.5):  # r (Z_i^0.23 + Z_j^0.23) in A
        ra, rb = x / ua, x / ub
        pa = _dimer_energy(sa, ra, [0, 1])[0][0] * ra / (Za[0] * Za[1])
        pb = _dimer_energy(sb, rb, [0, 1])[0][0] * rb / (Zb[0] * Zb[1])
        assert abs(pa - pb) < 1e-12 * abs(pa)
    s = zbl_spec((26.0, 26.0), r1=1.2, r2=1.8)
    assert _dimer_energy(s, 1.8, [0, 0])[0][0] == 0.0
    assert _dimer_energy(s, 2.5, [0, 0])[0][0] == 0.0
    e_in = [_dimer_energy(s, r, [0, 0])[0][0] for r in (1.79999, 1.8 - 2e-5)]
    assert 0.0 < e_in[0] < e_in[1] < 1e-6  # vanishes quadratically at r2
    # at r < r1 the switch is 1: the energy equals the unswitched one of a wider switch
    wide = zbl_spec((26.0, 26.0), r1=1.5, r2=1.9)
    assert _dimer_energy(s, 1.1, [0, 0])[0][0] == _dimer_energy(wide, 1.1, [0, 0])[0][0]


def test_zbl_forces_and_virial_finite_difference():
    """F = -dE/dr and W = -dE/d(eps) with the ZBL term on, on a compressed two-species cell
    where many pairs fall inside the switch region and inside r1."""
    s = zbl_spec((14.0, 6.0), r1=1.2, r2=2.2)
    rng = np.random.default_rng(3)
    cell = np.eye(3) * 4.2 + 0.1 * rng.uniform(-1, 1, (3, 3))
    pos = rng.uniform(0, 1, (9, 3)) @ cell
    b = fd_batch(one_batch(pos, cell, rng.integers(0, 2, 9)))
    theta = synth.random_theta(oracle.num_params(s), 4)
    qs = oracle.scale_from_range(oracle.descriptors(s, theta, b))
    E, F, W = oracle.evaluate(s, theta, qs, b)
    E0 = oracle.evaluate(zbl_spec_off(s), theta, qs, b)[0]
    assert abs(E[0] - E0[0]) > 1.0  # the ZBL term is a large part of this cell's energy
    h = 1e-6
    for i in range(b.n_atoms):
        for a in range(3):
            bp, bm = fd_batch(b), fd_batch(b)
            bp.pos[i, a] += h
            bm.pos[i, a] -= h
            fd = -(oracle.evaluate(s, theta, qs, bp)[0][0] - oracle.evaluate(s, theta, qs, bm)[0][0]) / (2 * h)
            assert abs(fd - F[i, a]) < 1e-6 * max(1.0, np.abs(F).max())
    for ab in range(9):
        eps = np.zeros(9)
        eps[ab] = h
        out = []
        for sgn in (1, -1):
            Fm = np.eye(3) + sgn * eps.reshape(3, 3)
            bb = fd_batch(b)
            bb.pos = bb.pos @ Fm.T
            bb.cell[0] = (bb.cell[0].reshape(3, 3) @ Fm.T).reshape(9)
            out.append(oracle.evaluate(s, theta, qs, bb)[0][0])
        assert abs(-(out[0] - out[1]) / (2 * h) - W[0, ab]) < 1e-6 * max(1.0, np.abs(W).max())
    assert np.allclose(F.sum(axis=0), 0.0, atol=1e-9)


def zbl_spec_off(s):
    t = Spec(**{k: v for k, v in s.__dict__.items() if k != "zbl"})
    return t


def test_zbl_leaves_the_parameter_gradient_to_the_network():
    """The ZBL term has no trainable parameter: the parameter gradient of a fixed-cotangent
    objective sum dE E + sum dF.F + sum dW:W does not change when it is switched on."""
    s = zbl_spec((14.0, 6.0), r1=1.2, r2=2.2)
    rng = np.random.default_rng(5)
    cell = np.eye(3) * 4.4
    pos = rng.uniform(0, 1, (8, 3)) @ cell
    b = one_batch(pos, cell, rng.integers(0, 2, 8))
    theta = synth.random_theta(oracle.num_params(s), 6)
    qs = oracle.scale_from_range(oracle.descriptors(s, theta, b))
    dE, dF, dW = rng.normal(size=1), rng.normal(size=(8, 3)), rng.normal(size=(1, 9))
    g_on = oracle.backward(s, theta, qs, b, dE, dF, dW)
    g_off = oracle.backward(zbl_spec_off(s), theta, qs, b, dE, dF, dW)
    assert np.array_equal(g_on, g_off)
