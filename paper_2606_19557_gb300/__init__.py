"""GB300-native NEP loss + parameter-gradient hot path (TorchNEP, arXiv 2606.19557).

Thin ctypes binding over ``libnep_gb300.so`` (the C ABI of ``include/nep_gb300.h``).
Every step of the computation runs in the library's CUDA kernels; PyTorch only
provides device memory and streams.  There is no CPU fallback: if the library is
missing or no GPU is present, calls raise.

    from paper_2606_19557_gb300 import NEP, synth
    spec = synth.SPECS["fcc_bcc_t1"]
    nep = NEP(spec)
    nep.set_structures_batch(synth.batch_fcc_bcc(n_struct=10))
    nep.set_params(theta, q_scale)             # float32 CUDA tensors
    E, F, W = nep.eval()
    loss3, grad = nep.loss_grad(E_ref, F_ref, W_ref, lam=(1.0, 1.0, 0.1))
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnep_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "nep_gb300.h")

NEP_OK, NEP_EINVAL, NEP_ENOMEM, NEP_ECUDA, NEP_ESTATE, NEP_EINTERNAL = 0, -1, -2, -3, -4, -5
SCHED_PERSISTENT, SCHED_PLAIN = 0, 1
KERNEL_COUNT = 10

_lib = None
_lock = threading.Lock()


class NepError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"NEP error {code}: {msg}")
        self.code = code


class OptimConfig(ctypes.Structure):
    """nep_optim_config: AMSGrad (paper defaults beta1 0.9, beta2 0.999, eps 1e-8) and the plateau schedule."""
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("factor", ctypes.c_double), ("patience", ctypes.c_int),
                ("lr_min", ctypes.c_double), ("threshold", ctypes.c_double)]


class _Config(ctypes.Structure):
    _fields_ = [("n_types", ctypes.c_int), ("rc_R", ctypes.c_float), ("rc_A", ctypes.c_float),
                ("n_max_R", ctypes.c_int), ("n_max_A", ctypes.c_int), ("basis_R", ctypes.c_int),
                ("basis_A", ctypes.c_int), ("l_max", ctypes.c_int), ("has_4b", ctypes.c_int),
                ("has_5b", ctypes.c_int), ("n_neuron", ctypes.c_int), ("precision", ctypes.c_int),
                ("device", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree for sm_103a."""
    from . import build_ext as _b
    return _b.build(force=force)


def declared_symbols() -> list:
    """Entry points declared in include/nep_gb300.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\**(nep_\w+)\s*\(", txt, re.M)))


def load_library():
    """Loads libnep_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2606_19557_gb300.build()")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "nep_create": (I, [ctypes.POINTER(_Config), P, ctypes.POINTER(P)]),
            "nep_destroy": (None, [P]),
            "nep_num_params": (I, [P, ctypes.POINTER(I64)]),
            "nep_num_descriptors": (I, [P, ctypes.POINTER(I)]),
            "nep_set_params": (I, [P, P, P]),
            "nep_set_structures": (I, [P, I64, P, P, P, P]),
            "nep_num_pairs": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
            "nep_update_positions": (I, [P, P, P]),
            "nep_set_skin": (I, [P, ctypes.c_float]),
            "nep_get_neighbors": (I, [P, P, P, P, P]),
            "nep_eval": (I, [P, P, P, P]),
            "nep_descriptors": (I, [P, P]),
            "nep_descriptor_range": (I, [P, P, P]),
            "nep_loss_grad": (I, [P, P, P, P, P, D, D, D, P, P]),
            "nep_backward": (I, [P, P, P, P, P]),
            "nep_set_zbl": (I, [P, ctypes.c_float, ctypes.c_float, P]),
            "nep_set_loss_normalizers": (I, [P, D, D, D]),
            "nep_set_targets": (I, [P, P, P, P, P]),
            "nep_loss_grad_host": (I, [P, P, D, D, D, P, P]),
            "nep_optim_init": (I, [P, ctypes.POINTER(OptimConfig)]),
            "nep_optim_step": (I, [P, P, P]),
            "nep_train_step": (I, [P, D, D, D, P]),
            "nep_optim_epoch_end": (I, [P]),
            "nep_optim_set_lr": (I, [P, D]),
            "nep_optim_state": (I, [P, P]),
            "nep_get_params": (I, [P, P]),
            "nep_minibatch_setup": (I, [P, I, ctypes.POINTER(I64)]),
            "nep_minibatch_loss_grad": (I, [P, I64, D, D, D, P, P]),
            "nep_minibatch_train_step": (I, [P, I64, D, D, D, P]),
            "nep_minibatch_epoch": (I, [P, P, I64, D, D, D]),
            "nep_set_schedule": (I, [P, I]),
            "nep_autotune": (I, [P]),
            "nep_get_launch": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
            "nep_set_launch": (I, [P, I, I, I, I]),
            "nep_get_variant": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
            "nep_set_variant": (I, [P, I, I]),
            "nep_set_timing": (I, [P, I]),
            "nep_kernel_times": (I, [P, P, ctypes.POINTER(I)]),
            "nep_kernel_name": (ctypes.c_char_p, [I]),
            "nep_last_error": (ctypes.c_char_p, [P]),
            "nep_fp32_fma_probe": (I, [P, I, I64, P, ctypes.POINTER(D)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(t) -> Optional[int]:
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class NEP:
    """One NEP model on one GPU: cached batch, parameters and a CUDA stream of its own.

    ``spec`` carries the model keys of the paper's input file (Table 1): n_types,
    rc_R, rc_A, n_max_R, n_max_A, basis_R, basis_A, l_max, has_4b, has_5b, n_neu.
    """

    def __init__(self, spec, device: int = 0):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.spec = spec
        self.device = torch.device("cuda", device)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.Stream(device=self.device)
        cfg = _Config(int(spec.n_types), float(spec.rc_R), float(spec.rc_A), int(spec.n_max_R), int(spec.n_max_A),
                      int(spec.basis_R), int(spec.basis_A), int(spec.l_max), int(spec.has_4b), int(spec.has_5b),
                      int(spec.n_neu), 0, int(device))
        h = ctypes.c_void_p()
        rc = self.lib.nep_create(ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != NEP_OK:
            raise NepError(rc, self.lib.nep_last_error(None).decode())
        self.h = h
        P = ctypes.c_int64()
        self.lib.nep_num_params(self.h, ctypes.byref(P))
        nd = ctypes.c_int()
        self.lib.nep_num_descriptors(self.h, ctypes.byref(nd))
        self.P, self.n_des = int(P.value), int(nd.value)
        self.n_struct = 0
        self.n_atoms = 0
        self._keep = []
        zbl = getattr(spec, "zbl", None)
        if zbl:
            self.set_zbl(*zbl)

    # ------------------------------------------------------------------ plumbing
    def _check(self, rc: int):
        if rc != NEP_OK:
            raise NepError(rc, self.lib.nep_last_error(self.h).decode())

    def _enter(self):
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def _leave(self):
        self.torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _call(self, fn, *args):
        self._enter()
        rc = fn(self.h, *args)
        self._leave()
        self._check(rc)

    def close(self):
        if getattr(self, "h", None):
            self.lib.nep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, x, dtype):
        t = self.torch
        if not isinstance(x, t.Tensor):
            x = t.as_tensor(x)
        return x.to(device=self.device, dtype=dtype).contiguous()

    # ------------------------------------------------------------------ model state
    def set_params(self, theta, q_scale):
        """theta [P] and normalisation factors q_scale [N_des] (Eq. "norm"), float32."""
        th = self._dev(theta, self.torch.float32).reshape(-1)
        qs = self._dev(q_scale, self.torch.float32).reshape(-1)
        if th.numel() != self.P or qs.numel() != self.n_des:
            raise ValueError(f"theta must have {self.P} entries and q_scale {self.n_des}")
        self._call(self.lib.nep_set_params, _ptr(th), _ptr(qs))
        self._keep = [th, qs]
        self.theta, self.q_scale = th, qs

    def set_structures(self, atom_off, pos, types, cell):
        """Caches a batch (CSR atom offsets, positions, species, cells) and builds its neighbour lists."""
        t = self.torch
        off = self._dev(atom_off, t.int64).reshape(-1)
        p = self._dev(pos, t.float32).reshape(-1, 3)
        ty = self._dev(types, t.int32).reshape(-1)
        c = self._dev(cell, t.float32).reshape(-1, 9)
        ns = off.numel() - 1
        self._call(self.lib.nep_set_structures, ns, _ptr(off), _ptr(p), _ptr(ty), _ptr(c))
        self.n_struct, self.n_atoms = ns, int(p.shape[0])
        self.atom_off = off

    def set_structures_batch(self, batch):
        """set_structures from an object with atom_off, pos, types and cell arrays."""
        self.set_structures(batch.atom_off, batch.pos, batch.types, batch.cell)

    def update_positions(self, pos, cell=None):
        """New positions (and cells) for the cached structures; rebuilds the neighbour lists."""
        t = self.torch
        p = self._dev(pos, t.float32).reshape(-1)
        cl = None if cell is None else self._dev(cell, t.float32).reshape(-1)
        if p.numel() != 3 * self.n_atoms or (cl is not None and cl.numel() != 9 * self.n_struct):
            raise ValueError("positions [N_a, 3] and cells [n_struct, 9] of the cached batch expected")
        self._call(self.lib.nep_update_positions, _ptr(p), _ptr(cl))

    def set_skin(self, skin: float):
        """Skin (Angstrom) of the candidate lists behind update_positions with the cells kept; 0 scans every time."""
        self._call(self.lib.nep_set_skin, float(skin))

    def num_pairs(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.nep_num_pairs(self.h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def neighbors(self):
        """(nbr_off [Na+1], j [M], shift [M,3], ang [M]) of the cached batch."""
        t = self.torch
        M, _ = self.num_pairs()
        off = t.empty(self.n_atoms + 1, dtype=t.int64, device=self.device)
        j = t.empty(max(M, 1), dtype=t.int32, device=self.device)
        s = t.empty(max(M, 1) * 3, dtype=t.int32, device=self.device)
        a = t.empty(max(M, 1), dtype=t.uint8, device=self.device)
        self._call(self.lib.nep_get_neighbors, _ptr(off), _ptr(j), _ptr(s), _ptr(a))
        return off, j[:M], s[:3 * M].reshape(M, 3), a[:M]

    # ------------------------------------------------------------------ hot path
    def eval(self):
        """(E [Ns] float64, F [Na,3] float32, W [Ns,9] float64) at the current parameters."""
        t = self.torch
        E = t.empty(max(self.n_struct, 1), dtype=t.float64, device=self.device)
        F = t.empty(max(self.n_atoms, 1), 3, dtype=t.float32, device=self.device)
        W = t.empty(max(self.n_struct, 1), 9, dtype=t.float64, device=self.device)
        self._call(self.lib.nep_eval, _ptr(E), _ptr(F), _ptr(W))
        return E[:self.n_struct], F[:self.n_atoms], W[:self.n_struct]

    def descriptors(self):
        t = self.torch
        q = t.empty(max(self.n_atoms, 1), self.n_des, dtype=t.float32, device=self.device)
        self._call(self.lib.nep_descriptors, _ptr(q))
        return q[:self.n_atoms]

    def descriptor_range(self):
        t = self.torch
        lo = t.empty(self.n_des, dtype=t.float32, device=self.device)
        hi = t.empty(self.n_des, dtype=t.float32, device=self.device)
        self._call(self.lib.nep_descriptor_range, _ptr(lo), _ptr(hi))
        return lo, hi

    def loss_grad(self, E_ref, F_ref, W_ref, has_W=None, lam: Sequence[float] = (1.0, 1.0, 0.1),
                  out=None):
        """Eq. "loss": returns (loss3 = (DE, DF, DV) float64 [3], dL/dtheta float32 [P])."""
        t = self.torch
        Er = self._dev(E_ref, t.float64).reshape(-1)
        Fr = self._dev(F_ref, t.float32).reshape(-1)
        Wr = self._dev(W_ref, t.float64).reshape(-1)
        hw = None if has_W is None else self._dev(has_W, t.uint8).reshape(-1)
        if out is None:
            loss3 = t.empty(3, dtype=t.float64, device=self.device)
            grad = t.empty(self.P, dtype=t.float32, device=self.device)
        else:
            loss3, grad = out
        self._call(self.lib.nep_loss_grad, _ptr(Er), _ptr(Fr), _ptr(Wr), _ptr(hw), float(lam[0]), float(lam[1]),
                   float(lam[2]), _ptr(loss3), _ptr(grad))
        self._refs = (Er, Fr, Wr, hw)
        return loss3, grad

    def set_zbl(self, r1: float, r2: float, Z=None):
        """ZBL short-range term with switch radii r1 < r2 and atomic numbers Z [n_types]
        (nep_set_zbl); r2 = 0 switches it off."""
        if r2 == 0:
            self._check(self.lib.nep_set_zbl(self.h, 0.0, 0.0, None))
            return
        z = (ctypes.c_float * len(Z))(*[float(x) for x in Z])
        self._check(self.lib.nep_set_zbl(self.h, float(r1), float(r2), ctypes.cast(z, ctypes.c_void_p)))

    def set_loss_normalizers(self, N_s: float = 0.0, N_a: float = 0.0, N_s_V: float = 0.0):
        """Global N_s, N_a, N_s^V for a shard of a larger batch (0 = this batch's own)."""
        self._check(self.lib.nep_set_loss_normalizers(self.h, float(N_s), float(N_a), float(N_s_V)))

    def backward(self, dE, dF, dW):
        """d/dtheta of dE.E + dF.F + dW:W, using the state of the latest eval()."""
        t = self.torch
        a = self._dev(dE, t.float64).reshape(-1)
        b = self._dev(dF, t.float32).reshape(-1)
        c = self._dev(dW, t.float64).reshape(-1)
        grad = t.empty(self.P, dtype=t.float32, device=self.device)
        self._call(self.lib.nep_backward, _ptr(a), _ptr(b), _ptr(c), _ptr(grad))
        return grad

    def set_targets(self, E_ref, F_ref, W_ref, has_W=None):
        t = self.torch
        Er = self._dev(E_ref, t.float64).reshape(-1)
        Fr = self._dev(F_ref, t.float32).reshape(-1)
        Wr = self._dev(W_ref, t.float64).reshape(-1)
        hw = None if has_W is None else self._dev(has_W, t.uint8).reshape(-1)
        self._call(self.lib.nep_set_targets, _ptr(Er), _ptr(Fr), _ptr(Wr), _ptr(hw))
        self._tg = (Er, Fr, Wr, hw)

    def loss_grad_host(self, theta_host, lam=(1.0, 1.0, 0.1), loss3_host=None, grad_host=None):
        """Host-buffer step: theta (host float32) in, (loss3, grad) host arrays out; synchronizes."""
        t = self.torch
        th = theta_host if isinstance(theta_host, t.Tensor) else t.as_tensor(theta_host)
        th = th.to(dtype=t.float32).contiguous()
        if loss3_host is None:
            loss3_host = t.empty(3, dtype=t.float64, pin_memory=True)
        if grad_host is None:
            grad_host = t.empty(self.P, dtype=t.float32, pin_memory=True)
        self._enter()
        rc = self.lib.nep_loss_grad_host(self.h, _ptr(th), float(lam[0]), float(lam[1]), float(lam[2]),
                                         _ptr(loss3_host), _ptr(grad_host))
        self._check(rc)
        return loss3_host, grad_host

    # ------------------------------------------------------------------ scheduling
    # ---------------------------------------------------------------- training loop (Sec. "Training")
    def optim_init(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                   factor: float = 0.5, patience: int = 5, lr_min: float = 0.0, threshold: float = 0.0):
        """AMSGrad state (moments zeroed, t = 0) and the plateau schedule, on the device."""
        cfg = OptimConfig(float(lr), float(beta1), float(beta2), float(eps), float(factor), int(patience),
                          float(lr_min), float(threshold))
        self._call(self.lib.nep_optim_init, ctypes.byref(cfg))

    def optim_step(self, grad, loss=None):
        """One AMSGrad step on the context's parameters; ``loss`` (device scalar) joins the epoch mean."""
        t = self.torch
        g = self._dev(grad, t.float32).reshape(-1)
        lo = None if loss is None else self._dev(loss, t.float64).reshape(-1)
        self._call(self.lib.nep_optim_step, _ptr(g), _ptr(lo))
        self._opt_refs = (g, lo)

    def train_step(self, lam: Sequence[float] = (1.0, 1.0, 0.1), loss3=None):
        """Loss + gradient at the current parameters, then the AMSGrad step (one graph).
        Returns loss3 (DE, DF, DV before the update), a float64 device tensor."""
        t = self.torch
        if loss3 is None:
            loss3 = t.empty(3, dtype=t.float64, device=self.device)
        self._call(self.lib.nep_train_step, float(lam[0]), float(lam[1]), float(lam[2]), _ptr(loss3))
        return loss3

    def optim_epoch_end(self):
        self._call(self.lib.nep_optim_epoch_end)

    def optim_set_lr(self, lr: float):
        """Stage start: learning rate set, plateau schedule restarted (moments kept)."""
        self._call(self.lib.nep_optim_set_lr, float(lr))

    def optim_state(self) -> dict:
        out = (ctypes.c_double * 6)()
        self._check(self.lib.nep_optim_state(self.h, out))
        keys = ("t", "lr", "best", "bad_epochs", "last_epoch_loss", "reductions")
        return {k: float(v) for k, v in zip(keys, out)}

    def get_params(self):
        t = self.torch
        th = t.empty(self.P, dtype=t.float32, device=self.device)
        self._call(self.lib.nep_get_params, _ptr(th))
        return th

    # ---------------------------------------------------------------- mini-batch mode
    def minibatch_setup(self, batch_size: int) -> int:
        """Groups of ``batch_size`` consecutive cached structures; returns the group count."""
        n = ctypes.c_int64()
        self._call(self.lib.nep_minibatch_setup, int(batch_size), ctypes.byref(n))
        self.n_minibatches = int(n.value)
        return self.n_minibatches

    def minibatch_loss_grad(self, m: int, lam: Sequence[float] = (1.0, 1.0, 0.1)):
        t = self.torch
        loss3 = t.empty(3, dtype=t.float64, device=self.device)
        grad = t.empty(self.P, dtype=t.float32, device=self.device)
        self._call(self.lib.nep_minibatch_loss_grad, int(m), float(lam[0]), float(lam[1]), float(lam[2]),
                   _ptr(loss3), _ptr(grad))
        return loss3, grad

    def minibatch_train_step(self, m: int, lam: Sequence[float] = (1.0, 1.0, 0.1), loss3=None):
        self._call(self.lib.nep_minibatch_train_step, int(m), float(lam[0]), float(lam[1]), float(lam[2]),
                   _ptr(loss3))
        return loss3

    def minibatch_epoch(self, order, lam: Sequence[float] = (1.0, 1.0, 0.1)):
        """One epoch over the groups in ``order`` (host sequence of indices), then the
        epoch boundary of the schedule; runs asynchronously on the context's stream."""
        import numpy as np
        o = np.ascontiguousarray(np.asarray(order, dtype=np.int64).reshape(-1))
        self._call(self.lib.nep_minibatch_epoch, o.ctypes.data_as(ctypes.c_void_p), int(o.size), float(lam[0]),
                   float(lam[1]), float(lam[2]))

    def set_schedule(self, mode: int):
        self._check(self.lib.nep_set_schedule(self.h, int(mode)))

    def autotune(self):
        self._call(self.lib.nep_autotune)
        return self.launch_shape()

    def launch_shape(self):
        v = [ctypes.c_int() for _ in range(4)]
        self._check(self.lib.nep_get_launch(self.h, *[ctypes.byref(x) for x in v]))
        return tuple(int(x.value) for x in v)

    def variant(self):
        """(forward lanes per atom, forward registers, adjoint lanes per atom, adjoint registers)."""
        v = [ctypes.c_int() for _ in range(4)]
        self._check(self.lib.nep_get_variant(self.h, *[ctypes.byref(x) for x in v]))
        return tuple(int(x.value) for x in v)

    def set_variant(self, fwd_var: int, adj_var: int):
        """Kernel variants (0-5): lanes per atom 8 for 0-1, 16 for 2-3, 32 for 4-5; even = 128
        registers per thread, odd = 96."""
        self._call(self.lib.nep_set_variant, int(fwd_var), int(adj_var))

    def set_launch(self, fwd_warps=0, fwd_blocks=0, adj_warps=0, adj_blocks=0):
        self._call(self.lib.nep_set_launch, int(fwd_warps), int(fwd_blocks), int(adj_warps), int(adj_blocks))

    def set_timing(self, on: bool):
        self._check(self.lib.nep_set_timing(self.h, 1 if on else 0))

    def kernel_times(self):
        """{kernel name: ms} of the latest timed nep_loss_grad (waits for it)."""
        arr = (ctypes.c_float * KERNEL_COUNT)()
        n = ctypes.c_int(KERNEL_COUNT)
        self._check(self.lib.nep_kernel_times(self.h, arr, ctypes.byref(n)))
        return {self.lib.nep_kernel_name(k).decode(): float(arr[k]) for k in range(n.value)}


def param_blocks(spec) -> dict:
    """Slices of theta (layout of include/nep_gb300.h) by parameter block: w0, b0 and w1 of
    each species, the shared b1, and c_R and c_A of each ordered species pair."""
    T, NN = int(spec.n_types), int(spec.n_neu)
    NR, KR = spec.n_max_R + 1, spec.basis_R + 1
    NA, KA = spec.n_max_A + 1, spec.basis_A + 1
    ND = NR + NA * (spec.l_max + spec.has_4b + spec.has_5b)
    out, o = {}, 0
    for name, size in (("w0", NN * ND), ("b0", NN), ("w1", NN)):
        for t in range(T):
            out[f"{name}[{t}]"] = slice(o, o + size)
            o += size
    out["b1"] = slice(o, o + 1)
    o += 1
    for name, size in (("cR", NR * KR), ("cA", NA * KA)):
        for a in range(T):
            for b in range(T):
                out[f"{name}[{a},{b}]"] = slice(o, o + size)
                o += size
    return out


def fp32_fma_probe(stream, blocks: int, iters: int, sink) -> float:
    """Queues the library's FP32 FMA throughput kernel on `stream` (a torch.cuda.Stream)
    and returns its floating-point operation count (nep_fp32_fma_probe)."""
    lib = load_library()
    fl = ctypes.c_double(0.0)
    rc = lib.nep_fp32_fma_probe(ctypes.c_void_p(stream.cuda_stream), int(blocks), int(iters),
                                ctypes.c_void_p(sink.data_ptr()), ctypes.byref(fl))
    if rc != NEP_OK:
        raise NepError(rc, "nep_fp32_fma_probe failed")
    return fl.value


class NEPFunction:
    """torch.autograd.Function: theta -> (E, F, W); backward takes dL/dE, dL/dF, dL/dW.

    The forward runs nep_eval, the backward the adjoint kernel (forward-mode JVP of the
    descriptors along dL/dF and dL/dW, then reverse mode through tanh' and tanh'' into
    the network weights and the c coefficients).  Use ``NEPFunction.apply(theta, nep)``.
    """

    _fn = None

    @classmethod
    def apply(cls, theta, nep: NEP):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, th, model):
                    model.set_params(th.detach(), model.q_scale)
                    E, F, W = model.eval()
                    ctx.model = model
                    return E, F, W

                @staticmethod
                def backward(ctx, gE, gF, gW):
                    m = ctx.model
                    t = torch
                    gE = t.zeros(m.n_struct, dtype=t.float64, device=m.device) if gE is None else gE
                    gF = t.zeros(m.n_atoms, 3, dtype=t.float32, device=m.device) if gF is None else gF
                    gW = t.zeros(m.n_struct, 9, dtype=t.float64, device=m.device) if gW is None else gW
                    return m.backward(gE, gF, gW), None

            cls._fn = _F
        return cls._fn.apply(theta, nep)


from . import synth  # noqa: E402  (geometry generator; no model arithmetic)

__all__ = ["NEP", "NEPFunction", "NepError", "build", "load_library", "declared_symbols", "synth",
           "SCHED_PERSISTENT", "SCHED_PLAIN"]
