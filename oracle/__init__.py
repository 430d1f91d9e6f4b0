"""FP64 CPU oracle for the NEP hot path.  TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It never imports the product package
and shares no code with the CUDA sources; it compiles ``nep_oracle.c`` with
gcc into ``oracle/_build/`` and calls it through ctypes.

Every function here takes and returns numpy arrays.  A ``batch`` is any object
with ``atom_off`` (int64 [Ns+1]), ``pos`` ([Na,3]), ``types`` (int32 [Na]) and
``cell`` ([Ns,9], rows = lattice vectors).  Positions and cells are used in FP64;
the pair-inclusion decision rounds them to float first, as the GPU path, which
receives float32 inputs, does.  A ``spec`` is any object with the model fields
of the paper's input file (Table 1): n_types, rc_R, rc_A, n_max_R, n_max_A,
basis_R, basis_A, l_max, has_4b, has_5b, n_neu.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nep_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libnep_oracle.so")
_lock = threading.Lock()
_lib = None


class _Cfg(ctypes.Structure):
    _fields_ = [("n_types", ctypes.c_int), ("rc_R", ctypes.c_double), ("rc_A", ctypes.c_double),
                ("n_max_R", ctypes.c_int), ("n_max_A", ctypes.c_int), ("basis_R", ctypes.c_int),
                ("basis_A", ctypes.c_int), ("l_max", ctypes.c_int), ("has_4b", ctypes.c_int),
                ("has_5b", ctypes.c_int), ("n_neu", ctypes.c_int), ("zbl", ctypes.c_int),
                ("zbl_r1", ctypes.c_double), ("zbl_r2", ctypes.c_double), ("zbl_Z", ctypes.c_double * 16)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP64, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            lib.orc_num_params.restype = ctypes.c_int64
            lib.orc_num_params.argtypes = [ctypes.POINTER(_Cfg)]
            lib.orc_num_descriptors.restype = ctypes.c_int
            lib.orc_num_descriptors.argtypes = [ctypes.POINTER(_Cfg)]
            lib.orc_neighbors.restype = ctypes.c_int64
            lib.orc_neighbors.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_int64,
                                          P, P, P, P]
            lib.orc_eval.restype = ctypes.c_int
            lib.orc_eval.argtypes = [ctypes.POINTER(_Cfg), P, P, ctypes.c_int64, P, P, P, P, P, P, P, P]
            lib.orc_backward.restype = ctypes.c_int
            lib.orc_backward.argtypes = [ctypes.POINTER(_Cfg), P, P, ctypes.c_int64, P, P, P, P, P, P, P, P]
            lib.orc_loss_grad.restype = ctypes.c_int
            lib.orc_loss_grad.argtypes = [ctypes.POINTER(_Cfg), P, P, ctypes.c_int64, P, P, P, P, P, P, P, P,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P, P, P, P]
            lib.orc_descriptors.restype = ctypes.c_int
            lib.orc_descriptors.argtypes = [ctypes.POINTER(_Cfg), P, ctypes.c_int64, P, P, P, P, P]
            lib.orc_ylm.restype = None
            lib.orc_ylm.argtypes = [P, ctypes.c_int, P, P]
            lib.orc_basis.restype = None
            lib.orc_basis.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P]
            lib.orc_kappa4.restype = ctypes.c_double
            lib.orc_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _cfg(spec) -> _Cfg:
    """The spec's model keys; an optional attribute zbl = (r1, r2, Z per species) adds the
    ZBL short-range term."""
    z = getattr(spec, "zbl", None)
    Z = (ctypes.c_double * 16)(*([float(x) for x in z[2]] if z else []))
    return _Cfg(int(spec.n_types), float(spec.rc_R), float(spec.rc_A), int(spec.n_max_R), int(spec.n_max_A),
                int(spec.basis_R), int(spec.basis_A), int(spec.l_max), int(spec.has_4b), int(spec.has_5b),
                int(spec.n_neu), 1 if z else 0, float(z[0]) if z else 0.0, float(z[1]) if z else 0.0, Z)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _arrays(batch):
    off = np.ascontiguousarray(batch.atom_off, dtype=np.int64)
    pos = np.ascontiguousarray(batch.pos, dtype=np.float64).reshape(-1, 3)
    typ = np.ascontiguousarray(batch.types, dtype=np.int32)
    cell = np.ascontiguousarray(batch.cell, dtype=np.float64).reshape(-1, 9)
    return off, pos, typ, cell


def threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all host cores)."""
    return int(_load().orc_threads())


def set_threads(n: int) -> None:
    """Threads for the following calls; n <= 0 restores one per host core."""
    lib = _load()
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_set_threads.restype = None
    lib.orc_set_threads(int(n))


def num_params(spec) -> int:
    return int(_load().orc_num_params(ctypes.byref(_cfg(spec))))


def num_descriptors(spec) -> int:
    return int(_load().orc_num_descriptors(ctypes.byref(_cfg(spec))))


def kappa4() -> float:
    return float(_load().orc_kappa4())


def neighbors(batch, rc_R: float, rc_A: float):
    """Brute-force pair list over all periodic images: (i, j, S [M,3], ang [M] bool)."""
    lib = _load()
    off, pos, _, cell = _arrays(batch)
    ns = off.shape[0] - 1
    dummy = np.zeros(1, np.int64)
    m = lib.orc_neighbors(ns, _p(off), _p(pos), _p(cell), rc_R, rc_A, 0, _p(dummy), _p(dummy),
                          _p(np.zeros(3, np.int32)), _p(np.zeros(1, np.uint8)))
    if m < 0:
        raise ValueError("degenerate cell")
    i = np.zeros(max(m, 1), np.int64)
    j = np.zeros(max(m, 1), np.int64)
    S = np.zeros((max(m, 1), 3), np.int32)
    ang = np.zeros(max(m, 1), np.uint8)
    lib.orc_neighbors(ns, _p(off), _p(pos), _p(cell), rc_R, rc_A, m, _p(i), _p(j), _p(S), _p(ang))
    return i[:m], j[:m], S[:m], ang[:m].astype(bool)


def evaluate(spec, theta, qscale, batch, want_q: bool = False):
    """E [Ns], F [Na,3], W [Ns,9] (and q [Na,ND] if asked) in FP64."""
    lib = _load()
    off, pos, typ, cell = _arrays(batch)
    ns, na = off.shape[0] - 1, int(off[-1])
    th = np.ascontiguousarray(theta, np.float64)
    qs = np.ascontiguousarray(qscale, np.float64)
    E = np.zeros(max(ns, 1))
    F = np.zeros((max(na, 1), 3))
    W = np.zeros((max(ns, 1), 9))
    nd = num_descriptors(spec)
    q = np.zeros((max(na, 1), nd)) if want_q else None
    c = _cfg(spec)
    rc = lib.orc_eval(ctypes.byref(c), _p(th), _p(qs), ns, _p(off), _p(pos), _p(typ), _p(cell), _p(E), _p(F), _p(W),
                      _p(q) if want_q else None)
    if rc != 0:
        raise ValueError(f"oracle eval failed ({rc})")
    out = (E[:ns], F[:na], W[:ns])
    return out + (q[:na],) if want_q else out


def descriptors(spec, theta, batch):
    """Raw descriptor vectors q [Na, ND] (before the normalisation of Eq. "norm")."""
    lib = _load()
    off, pos, typ, cell = _arrays(batch)
    ns, na = off.shape[0] - 1, int(off[-1])
    q = np.zeros((max(na, 1), num_descriptors(spec)))
    c = _cfg(spec)
    rc = lib.orc_descriptors(ctypes.byref(c), _p(np.ascontiguousarray(theta, np.float64)), ns, _p(off), _p(pos),
                             _p(typ), _p(cell), _p(q))
    if rc != 0:
        raise ValueError(f"oracle descriptors failed ({rc})")
    return q[:na]


def scale_from_range(q: np.ndarray) -> np.ndarray:
    """Eq. "norm" factors 1/(q_max - q_min) over a set of descriptors (1 where max == min)."""
    if q.shape[0] == 0:
        return np.ones(q.shape[1])
    span = q.max(axis=0) - q.min(axis=0)
    return np.where(span > 0, 1.0 / np.where(span > 0, span, 1.0), 1.0)


def loss_grad(spec, theta, qscale, batch, E_ref, F_ref, W_ref, has_W=None, lam=(1.0, 1.0, 0.1), norms=None):
    """Eq. "loss" terms (DE, DF, DV), dL/dtheta [P], and E, F, W, all FP64."""
    lib = _load()
    off, pos, typ, cell = _arrays(batch)
    ns, na = off.shape[0] - 1, int(off[-1])
    P = num_params(spec)
    Er = np.ascontiguousarray(E_ref, np.float64).reshape(-1)
    Fr = np.ascontiguousarray(F_ref, np.float64).reshape(-1)
    Wr = np.ascontiguousarray(W_ref, np.float64).reshape(-1)
    hw = None if has_W is None else np.ascontiguousarray(has_W, np.uint8)
    nr = None if norms is None else np.ascontiguousarray(norms, np.float64)
    loss3 = np.zeros(3)
    grad = np.zeros(P)
    E = np.zeros(max(ns, 1))
    F = np.zeros((max(na, 1), 3))
    W = np.zeros((max(ns, 1), 9))
    c = _cfg(spec)
    rc = lib.orc_loss_grad(ctypes.byref(c), _p(np.ascontiguousarray(theta, np.float64)),
                           _p(np.ascontiguousarray(qscale, np.float64)), ns, _p(off), _p(pos), _p(typ), _p(cell),
                           _p(Er), _p(Fr), _p(Wr), _p(hw) if hw is not None else None,
                           float(lam[0]), float(lam[1]), float(lam[2]), _p(nr) if nr is not None else None,
                           _p(loss3), _p(grad), _p(E), _p(F), _p(W))
    if rc != 0:
        raise ValueError(f"oracle loss_grad failed ({rc})")
    return loss3, grad, E[:ns], F[:na], W[:ns]


def backward(spec, theta, qscale, batch, dE, dF, dW):
    """Gradient of sum dE.E + sum dF.F + sum dW:W with respect to theta (FP64)."""
    lib = _load()
    off, pos, typ, cell = _arrays(batch)
    ns = off.shape[0] - 1
    grad = np.zeros(num_params(spec))
    c = _cfg(spec)
    rc = lib.orc_backward(ctypes.byref(c), _p(np.ascontiguousarray(theta, np.float64)),
                          _p(np.ascontiguousarray(qscale, np.float64)), ns, _p(off), _p(pos), _p(typ), _p(cell),
                          _p(np.ascontiguousarray(dE, np.float64).reshape(-1)),
                          _p(np.ascontiguousarray(dF, np.float64).reshape(-1)),
                          _p(np.ascontiguousarray(dW, np.float64).reshape(-1)), _p(grad))
    if rc != 0:
        raise ValueError(f"oracle backward failed ({rc})")
    return grad


def loss_value(loss3, lam) -> float:
    return float(lam[0] * loss3[0] + lam[1] * loss3[1] + lam[2] * loss3[2])


def ylm(d, lmax: int = 4):
    """Orthonormal real harmonics of d/|d| (l = 1..lmax) and their gradients with respect to d."""
    lib = _load()
    d = np.ascontiguousarray(d, np.float64)
    v = np.zeros(24)
    g = np.zeros(72)
    lib.orc_ylm(_p(d), lmax, _p(v), _p(g))
    L3 = lmax * (lmax + 2)
    return v[:L3], g.reshape(24, 3)[:L3]


def basis(r: float, rc: float, K: int):
    """f_k(r) and df_k/dr for k = 0..K-1 (Chebyshev basis times the cutoff function)."""
    lib = _load()
    f = np.zeros(K)
    fp = np.zeros(K)
    lib.orc_basis(float(r), float(rc), int(K), _p(f), _p(fp))
    return f, fp
