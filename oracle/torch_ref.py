"""Second FP64 reference: the NEP model in plain PyTorch float64 with autograd.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).

It differs from the C oracle in every step that could hide a derivation error:
  * forces F = -dE/dr and the virial W = -dE/d(eps) come from autograd with
    create_graph=True, and the parameter gradient of the E/F/W loss from a
    second backward pass ("double backward", the paper's autograd variant,
    Sec. "Training efficiency ...");
  * the 3-body invariants use the addition theorem instead of harmonics:
    q_nl = (2l+1)/(4 pi) sum_j sum_k g_n(r_ij) g_n(r_ik) P_l(cos theta_jik),
    which equals sum_m A_nlm^2 for orthonormal real Y_lm (Methods, Eq. "q3b");
  * P_l by Bonnet's recurrence, Chebyshev T_k by the trigonometric form
    T_k(x) = cos(k arccos x).
The 4-body term is KAPPA tr(M^3) with M = sum_j g_n (r^ r^T - I/3) and the
5-body term (q_n1)^2, the readings stated in the C oracle's header.
Pairs (i, j, S) are taken as input, so this module only checks the physics.
Sized for small cases (every angular pair-of-pairs is materialised).
"""
from __future__ import annotations

import math

import numpy as np
import torch

KAPPA = -4.5 * math.sqrt(2.0 / 35.0) * (5.0 / (4.0 * math.pi)) ** 1.5


def _sizes(spec):
    NR, KR = spec.n_max_R + 1, spec.basis_R + 1
    NA, KA = spec.n_max_A + 1, spec.basis_A + 1
    L = spec.l_max
    ND = NR + NA * (L + spec.has_4b + spec.has_5b)
    return NR, KR, NA, KA, L, ND


def _split_theta(spec, th):
    NR, KR, NA, KA, L, ND = _sizes(spec)
    T, NN = spec.n_types, spec.n_neu
    o = 0
    w0 = th[o:o + T * NN * ND].reshape(T, NN, ND); o += T * NN * ND
    b0 = th[o:o + T * NN].reshape(T, NN); o += T * NN
    w1 = th[o:o + T * NN].reshape(T, NN); o += T * NN
    b1 = th[o]; o += 1
    cR = th[o:o + T * T * NR * KR].reshape(T, T, NR, KR); o += T * T * NR * KR
    cA = th[o:o + T * T * NA * KA].reshape(T, T, NA, KA); o += T * T * NA * KA
    assert o == th.shape[0]
    return w0, b0, w1, b1, cR, cA


def _basis(r, rc, K):
    """f_k(r) = 1/2 (T_k(x) + 1) f_c(r), x = 2 (r/rc - 1)^2 - 1, T_k(x) = cos(k arccos x)."""
    fc = torch.where(r <= rc, 0.5 * (torch.cos(math.pi * r / rc) + 1.0), torch.zeros_like(r))
    x = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    # arccos has an infinite derivative at |x| = 1 (r = 0 or r = rc); clamp stays inside for real pairs
    t = torch.arccos(torch.clamp(x, -1.0 + 1e-15, 1.0 - 1e-15))
    k = torch.arange(K, dtype=r.dtype)
    T = torch.cos(k[None, :] * t[:, None])
    return 0.5 * (T + 1.0) * fc[:, None]


def _legendre(x, L):
    P = [torch.ones_like(x), x]
    for l in range(1, L):
        P.append(((2 * l + 1) * x * P[l] - l * P[l - 1]) / (l + 1))
    return P


def energy_fn(spec, batch, pairs, theta, qscale):
    """Returns a function (pos, eps) -> (E_s [Ns], q [Na,ND]) with autograd through everything."""
    NR, KR, NA, KA, L, ND = _sizes(spec)
    off = np.asarray(batch.atom_off, np.int64)
    ns, na = off.shape[0] - 1, int(off[-1])
    sid = np.repeat(np.arange(ns), np.diff(off))
    types = torch.as_tensor(np.asarray(batch.types, np.int64))
    cell = torch.as_tensor(np.asarray(batch.cell, np.float64).reshape(ns, 3, 3))
    pi_, pj_, pS, pang = pairs
    pi = torch.as_tensor(np.asarray(pi_, np.int64))
    pj = torch.as_tensor(np.asarray(pj_, np.int64))
    S = torch.as_tensor(np.asarray(pS, np.float64))
    ang = np.asarray(pang, bool)
    psid = torch.as_tensor(sid[np.asarray(pi_, np.int64)])
    qs = torch.as_tensor(np.asarray(qscale, np.float64))
    ai = np.nonzero(ang)[0]
    # angular pair-of-pairs (p1, p2) sharing the centre atom, p1 == p2 included
    by_atom = {}
    for p in ai:
        by_atom.setdefault(int(pi_[p]), []).append(p)
    pp1, pp2 = [], []
    for lst in by_atom.values():
        for a in lst:
            for b in lst:
                pp1.append(a)
                pp2.append(b)
    pp1 = torch.as_tensor(np.asarray(pp1, np.int64))
    pp2 = torch.as_tensor(np.asarray(pp2, np.int64))
    ai_t = torch.as_tensor(ai)

    def f(th, pos, eps):
        w0, b0, w1, b1, cR, cA = _split_theta(spec, th)
        Fm = torch.eye(3, dtype=torch.float64)[None] + eps  # r -> (I + eps) r for atoms and cell
        posd = torch.einsum("iab,ib->ia", Fm[torch.as_tensor(sid)], pos)
        celld = torch.einsum("sab,skb->ska", Fm, cell)
        d = posd[pj] + torch.einsum("pk,pka->pa", S, celld[psid]) - posd[pi]
        r = torch.sqrt((d * d).sum(-1))
        ti, tj = types[pi], types[pj]
        fR = _basis(r, spec.rc_R, KR)
        gR = torch.einsum("pk,pnk->pn", fR, cR[ti, tj])
        q = [torch.zeros(na, NR, dtype=torch.float64).index_add(0, pi, gR)]
        if NA > 0 and (L > 0 or spec.has_4b or spec.has_5b):
            ra, da = r[ai_t], d[ai_t]
            fA = _basis(ra, spec.rc_A, KA)
            gA = torch.einsum("pk,pnk->pn", fA, cA[ti[ai_t], tj[ai_t]])
            u = da / ra[:, None]
            g_full = torch.zeros(r.shape[0], NA, dtype=torch.float64).index_copy(0, ai_t, gA)
            u_full = torch.zeros(r.shape[0], 3, dtype=torch.float64).index_copy(0, ai_t, u)
            cos = (u_full[pp1] * u_full[pp2]).sum(-1)
            Pl = _legendre(cos, max(L, 1))
            gg = g_full[pp1] * g_full[pp2]
            q3 = []
            for l in range(1, L + 1):
                v = (2 * l + 1) / (4 * math.pi) * gg * Pl[l][:, None]
                q3.append(torch.zeros(na, NA, dtype=torch.float64).index_add(0, pi[pp1], v))
            q += q3
            if spec.has_4b:
                Q = u[:, :, None] * u[:, None, :] - torch.eye(3, dtype=torch.float64)[None] / 3.0
                M = torch.zeros(na, NA, 3, 3, dtype=torch.float64).index_add(0, pi[ai_t], gA[:, :, None, None] * Q[:, None])
                M3 = M @ M @ M
                q.append(KAPPA * (M3[..., 0, 0] + M3[..., 1, 1] + M3[..., 2, 2]))
            if spec.has_5b:
                q.append(q3[0] ** 2)
        qv = torch.cat(q, dim=1)
        qt = qv * qs[None]
        z = torch.einsum("imn,in->im", w0[types], qt) - b0[types]
        Ei = (w1[types] * torch.tanh(z)).sum(-1) - b1
        Es = torch.zeros(ns, dtype=torch.float64).index_add(0, torch.as_tensor(sid), Ei)
        return Es, qv

    return f


def evaluate(spec, batch, pairs, theta, qscale):
    """E [Ns], F [Na,3], W [Ns,9] via autograd (float64)."""
    f = energy_fn(spec, batch, pairs, theta, qscale)
    th = torch.as_tensor(np.asarray(theta, np.float64))
    pos = torch.as_tensor(np.asarray(batch.pos, np.float64)).requires_grad_(True)
    ns = np.asarray(batch.atom_off).shape[0] - 1
    eps = torch.zeros(ns, 3, 3, dtype=torch.float64, requires_grad=True)
    E, _ = f(th, pos, eps)
    gpos, geps = torch.autograd.grad(E.sum(), (pos, eps))
    return E.detach().numpy(), (-gpos).numpy(), (-geps).reshape(ns, 9).numpy()


def loss_grad(spec, batch, pairs, theta, qscale, E_ref, F_ref, W_ref, has_W=None, lam=(1.0, 1.0, 0.1)):
    """Eq. "loss" and its parameter gradient by double backward (float64)."""
    f = energy_fn(spec, batch, pairs, theta, qscale)
    off = np.asarray(batch.atom_off, np.int64)
    ns, na = off.shape[0] - 1, int(off[-1])
    cnt = torch.as_tensor(np.diff(off).astype(np.float64))
    th = torch.as_tensor(np.asarray(theta, np.float64)).clone().requires_grad_(True)
    pos = torch.as_tensor(np.asarray(batch.pos, np.float64)).requires_grad_(True)
    eps = torch.zeros(ns, 3, 3, dtype=torch.float64, requires_grad=True)
    E, _ = f(th, pos, eps)
    gpos, geps = torch.autograd.grad(E.sum(), (pos, eps), create_graph=True)
    F = -gpos
    W = -geps.reshape(ns, 9)
    Er = torch.as_tensor(np.asarray(E_ref, np.float64))
    Fr = torch.as_tensor(np.asarray(F_ref, np.float64)).reshape(na, 3)
    Wr = torch.as_tensor(np.asarray(W_ref, np.float64)).reshape(ns, 9)
    hw = torch.ones(ns, dtype=torch.float64) if has_W is None else torch.as_tensor(np.asarray(has_W, np.float64))
    nsv = float(hw.sum())
    dE = (((E - Er) / cnt) ** 2).sum() / ns
    dF = ((F - Fr) ** 2).sum() / (3.0 * na)
    dV = ((((W - Wr) / cnt[:, None]) ** 2).sum(-1) * hw).sum() / (9.0 * nsv) if nsv > 0 else torch.zeros((), dtype=torch.float64)
    Ltot = lam[0] * dE + lam[1] * dF + lam[2] * dV
    (g,) = torch.autograd.grad(Ltot, th)
    return np.array([dE.item(), dF.item(), float(dV.detach())]), g.numpy()
