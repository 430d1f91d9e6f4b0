"""Algorithmic FP32 arithmetic of one loss + gradient pass, per kernel.

Counts the floating-point operations of the algorithm the kernels implement (FMA = 2,
a transcendental or square root = 1), from the model sizes and the pair/atom counts of
a batch.  It is the numerator of the roofline fraction: achieved = flops / kernel time.

Per radial pair (K = K_R, N = N_R):
  forward descriptors : distance (7), basis values (4K + 8), and the species sum (K) for
            one species or g_n = sum_k c f_k (2NK) for several
  forward pair gradients : basis + derivatives (9K + 10), sum_k beta_k f'_k (2K), pair
            gradient (4), force/virial accumulation (21), distance (7)
  adjoint JVP : lambda_p (24), distance (7), r^.lambda (6), basis + derivatives (9K + 10),
            two species sums (3K)                                          -> 12K + 47
Per angular pair (K = K_A, N = N_A, L3 = 24):
  forward descriptors : distance, basis, g_n = sum_k c f_k (2NK), 24 harmonics (72),
            moments (2 N L3)
  forward pair gradients : distance, basis + derivatives, g and g' (4NK), harmonics +
            gradients (172), dE/dA contractions (4 N L3), force assembly (8 L3 + 36)
  adjoint JVP : lambda / distance / basis / harmonics (9K + 225), g and g' (4NK), the
            projected gradients (6 L3) and the JVP of the moments (4 N L3)
  adjoint coefficient gradient : lambda / distance / basis / harmonics again (9K + 225),
            alpha/beta (6 N L3 + 6 L3), coefficient terms (4NK)
Per atom: descriptor contractions and invariants, the network forward (4 N_des N_neu:
z = W0 q~ and b = W0^T u), the network reverse pass (4 N_des N_neu: v = W0 dq~ and
abar = W0^T zeta), dE/dA, beta, dJ/dA and the radial coefficient gradient, and
the network-gradient contraction (4 N_des N_neu).
"""
from __future__ import annotations

L3 = 24


def _sizes(spec):
    NR, KR = spec.n_max_R + 1, spec.basis_R + 1
    NA, KA = spec.n_max_A + 1, spec.basis_A + 1
    ND = NR + NA * (spec.l_max + spec.has_4b + spec.has_5b)
    return NR, KR, NA, KA, ND, spec.n_neu, spec.n_types


def per_unit(spec) -> dict:
    NR, KR, NA, KA, ND, NN, T = _sizes(spec)
    rad_desc = KR if T == 1 else 2 * NR * KR
    return {
        "desc_radial_pair": 7 + 4 * KR + 8 + rad_desc,
        "desc_angular_pair": 7 + 4 * KA + 8 + 2 * NA * KA + 72 + 2 * NA * L3,
        "desc_atom": (2 * T * KR * NR if T == 1 else 0) + 2 * L3 * NA + 70 * NA,
        "netfwd_atom": 4 * ND * NN + 6 * NN,
        "pair_radial_pair": 9 * KR + 10 + 2 * KR + 4 + 21 + 7,
        "pair_angular_pair": 7 + 9 * KA + 10 + 4 * NA * KA + 172 + 4 * NA * L3 + 8 * L3 + 36,
        "pair_atom": 4 * NA * L3 + 60 * NA + 2 * T * KR * NR,
        "jvp_radial_pair": 12 * KR + 47,
        "jvp_angular_pair": (24 + 7 + 12 + 9 * KA + 10 + 72 + 100) + 4 * NA * KA + NA + 6 * L3 + 4 * NA * L3,
        "jvp_atom": 2 * T * KR * NR + 4 * NA * L3 + 60 * NA,
        "netrev_atom": 4 * ND * NN + 12 * NN,
        "cg_angular_pair": (24 + 7 + 12 + 9 * KA + 10 + 72 + 100) + 6 * L3 + 6 * NA * L3 + 4 * NA * KA,
        "cg_atom": 60 * NA + 8 * NA * L3 + 4 * T * NR * KR,
        "net_atom": 4 * ND * NN + 2 * NN,
    }


def per_kernel(spec, n_atoms: int, n_radial: int, n_angular: int) -> dict:
    """Flops of one launch of each kernel (stage) of the pass; the angular pairs are a
    subset of the radial ones and count in both per-pair terms where both apply."""
    u = per_unit(spec)
    out = {
        "forward_desc": u["desc_radial_pair"] * n_radial + u["desc_angular_pair"] * n_angular
        + u["desc_atom"] * n_atoms,
        "net_forward": u["netfwd_atom"] * n_atoms,
        "forward_pair": u["pair_radial_pair"] * n_radial + u["pair_angular_pair"] * n_angular
        + u["pair_atom"] * n_atoms,
        "adjoint_jvp": u["jvp_radial_pair"] * n_radial + u["jvp_angular_pair"] * n_angular + u["jvp_atom"] * n_atoms,
        "net_reverse": u["netrev_atom"] * n_atoms,
        "adjoint_cgrad": u["cg_angular_pair"] * n_angular + u["cg_atom"] * n_atoms,
        "net_grad": u["net_atom"] * n_atoms,
    }
    out["forward"] = out["forward_desc"] + out["net_forward"] + out["forward_pair"]
    out["adjoint"] = out["adjoint_jvp"] + out["net_reverse"] + out["adjoint_cgrad"]
    return out
